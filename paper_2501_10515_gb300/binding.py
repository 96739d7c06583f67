"""ctypes binding of include/ascc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libascc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ascc.h")

ASCC_FP64 = 0
ASCC_MIXED_BF16 = 1
ASCC_FP64_TC = 2

STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "not converged", 5: "diverged", 6: "device wait timed out"}


class Excitation(C.Structure):
    _fields_ = [("n_csf", C.c_int32), ("hole", C.c_int32), ("particle", C.c_int32),
                ("beta", C.c_double), ("alpha", C.c_double), ("ansatz", C.c_int32),
                ("reserved", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("linearize", C.c_int32), ("triples", C.c_int32),
                ("pl_hole", C.c_int32), ("pl_particle", C.c_int32), ("r_tol", C.c_double),
                ("e_tol", C.c_double), ("max_iter", C.c_int32), ("diis_dim", C.c_int32),
                ("diis_start", C.c_int32), ("polish_iter", C.c_int32), ("polish_tol", C.c_double),
                ("ladder_stream", C.c_int32), ("reserved2", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("energy", C.c_double), ("e_ref", C.c_double), ("max_resid", C.c_double),
                ("iterations", C.c_int32), ("status", C.c_int32), ("iterations_low", C.c_int32),
                ("fp64_evaluations", C.c_int32)]


class TwoAnsatzResult(C.Structure):
    _fields_ = [("energy", C.c_double), ("converged", C.c_int32), ("reserved", C.c_int32),
                ("first", Result), ("second", Result)]


class Profile(C.Structure):
    _fields_ = [("ladder_ms", C.c_double), ("ladder_flops", C.c_double),
                ("ladder_launches", C.c_int64), ("launches", C.c_int64),
                ("gemm_flops", C.c_double), ("ladder_mma_flops", C.c_double)]


class ServeResult(C.Structure):
    _fields_ = [("request_id", C.c_int64), ("state_index", C.c_int32), ("status", C.c_int32),
                ("energy", C.c_double), ("iterations", C.c_int32), ("worker", C.c_int32),
                ("t_arrival", C.c_double), ("t_start", C.c_double), ("t_end", C.c_double)]


class AsccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
P = C.POINTER
dp = P(C.c_double)


def load():
    """Loads libascc.so (built by __graft_entry__.build / paper_2501_10515_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libascc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "ascc_default_options": (C.c_int, [P(Options)]),
        "ascc_create": (C.c_int, [P(vp), C.c_int32, C.c_int32, C.c_int32, dp, vp, C.c_int32,
                                  P(Excitation), P(Options), vp]),
        "ascc_create_sibling": (C.c_int, [P(vp), vp, P(Excitation), P(Options), vp]),
        "ascc_t3p_size": (C.c_int64, [vp]),
        "ascc_t3p_indices": (C.c_int, [vp, P(C.c_int32)]),
        "ascc_residual": (C.c_int, [vp, dp, dp, dp, dp, dp, dp, dp]),
        "ascc_residual_device": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "ascc_energy": (C.c_int, [vp, dp, dp, dp]),
        "ascc_solve": (C.c_int, [vp, P(Result)]),
        "ascc_solve_two_ansatz": (C.c_int, [vp, P(TwoAnsatzResult)]),
        "ascc_checkpoint_size": (C.c_int, [vp, P(C.c_int64)]),
        "ascc_checkpoint_save": (C.c_int, [vp, vp, C.c_int64]),
        "ascc_checkpoint_load": (C.c_int, [vp, vp, C.c_int64]),
        "ascc_reset": (C.c_int, [vp]),
        "ascc_iterate": (C.c_int, [vp, C.c_int32, P(Result)]),
        "ascc_set_profiling": (C.c_int, [vp, C.c_int32]),
        "ascc_get_profile": (C.c_int, [vp, P(Profile)]),
        "ascc_gemm_split_bf16": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_double,
                                           vp, vp, C.c_double, vp, vp]),
        "ascc_gemm_split_bf16_tiled": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                                 C.c_double, vp, vp, C.c_double, vp, vp,
                                                 C.c_int32]),
        "ascc_autotuned_classes": (C.c_int64, []),
        "ascc_selftest_bounded_wait": (C.c_int, [C.c_int32, vp]),
        "ascc_t3p_plan_check": (C.c_int64, [C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                            C.c_int32]),
        "ascc_gemm_fp64_tc": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_double, vp, vp,
                                        C.c_double, vp, vp]),
        "ascc_gemm_split_bf16_noalloc": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                                   C.c_double, vp, vp, C.c_double, vp, vp]),
        "ascc_server_create": (C.c_int, [P(vp), C.c_size_t, C.c_int32, P(Options)]),
        "ascc_server_submit": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, dp, dp, C.c_int32,
                                         P(Excitation), P(C.c_int64)]),
        "ascc_server_drain": (C.c_int, [vp]),
        "ascc_server_result_count": (C.c_int64, [vp]),
        "ascc_server_results": (C.c_int, [vp, P(ServeResult), C.c_int64]),
        "ascc_server_destroy": (None, [vp]),
        "ascc_get_state": (C.c_int, [vp, dp, dp, dp]),
        "ascc_set_state": (C.c_int, [vp, dp, dp, dp]),
        "ascc_footprint_bytes": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, P(Options)]),
        "ascc_launch_count": (C.c_int64, [vp]),
        "ascc_destroy": (None, [vp]),
        "ascc_status_string": (C.c_char_p, [C.c_int]),
        "ascc_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def symbols():
    """Function names declared in include/ascc.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(ascc_[a-z0-9_]+)\s*\(", text)))


def _check(st):
    if st != 0:
        raise AsccError(st, load().ascc_last_error().decode())


def gemm_split_bf16(A, B, out, level, alpha=1.0, beta=0.0, stream=None, tile=None):
    """out = alpha A B^T + beta out on device FP64 tensors (split-BF16 tensor cores);
    tile: None (the size rules) or the tile shape of ascc_gemm_split_bf16_tiled."""
    M, K = A.shape
    N = B.shape[0]
    assert tuple(out.shape) == (M, N) and B.shape[1] == K
    st = C.c_void_p(stream) if stream else None
    if tile is None:
        _check(load().ascc_gemm_split_bf16(M, N, K, level, alpha, C_void(A), C_void(B), beta,
                                           C_void(out), st))
    else:
        _check(load().ascc_gemm_split_bf16_tiled(M, N, K, level, alpha, C_void(A), C_void(B),
                                                 beta, C_void(out), st, int(tile)))


def selftest_bounded_wait(limit_ms=100, stream=None):
    """Status of a bounded device wait that cannot complete (ASCC_ERR_TIMEOUT expected)."""
    return int(load().ascc_selftest_bounded_wait(int(limit_ms),
                                                C.c_void_p(stream) if stream else None))


def t3p_plan_check(o, v, naux, nstreams, mode=0):
    """Unordered conflicting op pairs of the T3' stream plan plus intermediates that
    share workspace while live (0: race-free and correctly placed); host only.
    mode 1 drops the plan's event waits, mode 2 places every intermediate at 0."""
    return int(load().ascc_t3p_plan_check(o, v, naux, nstreams, int(mode)))


def autotuned_classes():
    """Shape classes the tile autotuner has timed in this process."""
    return int(load().ascc_autotuned_classes())


def gemm_fp64_tc(A, B, out, alpha=1.0, beta=0.0, stream=None):
    """out = alpha A B^T + beta out on device FP64 tensors (exact digit-plane
    products on the tensor cores, see ascc_gemm_fp64_tc)."""
    M, K = A.shape
    N = B.shape[0]
    assert tuple(out.shape) == (M, N) and B.shape[1] == K
    _check(load().ascc_gemm_fp64_tc(M, N, K, alpha, C_void(A), C_void(B), beta, C_void(out),
                                    C.c_void_p(stream) if stream else None))


def gemm_split_bf16_noalloc(A, B, out, level, alpha=1.0, beta=0.0, stream=None):
    """As gemm_split_bf16, with the operand planes in the library's fixed device
    scratch instead of newly allocated memory (see ascc_gemm_split_bf16_noalloc)."""
    M, K = A.shape
    N = B.shape[0]
    assert tuple(out.shape) == (M, N) and B.shape[1] == K
    _check(load().ascc_gemm_split_bf16_noalloc(M, N, K, level, alpha, C_void(A), C_void(B), beta,
                                               C_void(out), C.c_void_p(stream) if stream else None))


def C_void(x):
    return C.c_void_p(x.data_ptr())


def default_options(**kw) -> Options:
    opt = Options()
    _check(load().ascc_default_options(C.byref(opt)))
    for k, v in kw.items():
        setattr(opt, k, v)
    return opt


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(dp)


class Context:
    """One ASCC state (ground or one-CSF excited) of one molecule on the current GPU."""

    def __init__(self, o, v, naux, eps, B, hole=None, particle=None, beta=0.0, options=None,
                 stream=None, base=None, alpha=0.0, ansatz=0, **opt_kw):
        lib = load()
        self.o, self.v, self.naux = o, v, naux
        opt = options if options is not None else default_options()
        for k, val in opt_kw.items():
            setattr(opt, k, val)
        exc = (Excitation(0, 0, 0, 0.0, 0.0, 0, 0) if hole is None
               else Excitation(1, hole, particle, beta, alpha, ansatz, 0))
        h = C.c_void_p()
        s = C.c_void_p(stream) if stream else None
        if base is not None:
            st = lib.ascc_create_sibling(C.byref(h), base._h, C.byref(exc), C.byref(opt), s)
            self._keep = base
        else:
            eps = np.ascontiguousarray(eps, dtype=np.float64)
            if hasattr(B, "data_ptr"):          # a device tensor
                bptr, on_dev = C.c_void_p(B.data_ptr()), 1
            else:
                B = np.ascontiguousarray(B, dtype=np.float64)
                bptr, on_dev = C.c_void_p(B.ctypes.data), 0
            st = lib.ascc_create(C.byref(h), o, v, naux, _ptr(eps), bptr, on_dev, C.byref(exc),
                                 C.byref(opt), s)
        _check(st)
        self._h = h
        self.options = opt

    def close(self):
        if getattr(self, "_h", None):
            load().ascc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_t3(self) -> int:
        return int(load().ascc_t3p_size(self._h))

    def t3_indices(self) -> np.ndarray:
        idx = np.zeros((self.n_t3, 6), dtype=np.int32)
        _check(load().ascc_t3p_indices(self._h, idx.ctypes.data_as(P(C.c_int32))))
        return idx

    def residual(self, t1, t2, t3=None):
        """(E, R1, R2, R3) for host amplitudes."""
        o, v = self.o, self.v
        t1 = np.ascontiguousarray(t1, np.float64); t2 = np.ascontiguousarray(t2, np.float64)
        r1 = np.zeros((o, v)); r2 = np.zeros((o, o, v, v)); r3 = np.zeros(self.n_t3)
        e = np.zeros(1)
        t3 = None if t3 is None else np.ascontiguousarray(t3, np.float64)
        _check(load().ascc_residual(self._h, _ptr(t1), _ptr(t2), _ptr(t3), _ptr(r1), _ptr(r2),
                                    _ptr(r3) if self.n_t3 else None, _ptr(e)))
        return float(e[0]), r1, r2, r3

    def residual_device(self, t1, t2, t3, r1, r2, r3, e):
        """Residual on device buffers (integers: device addresses, or tensors)."""
        a = lambda x: None if x is None else C.c_void_p(x.data_ptr() if hasattr(x, "data_ptr") else x)
        _check(load().ascc_residual_device(self._h, a(t1), a(t2), a(t3), a(r1), a(r2), a(r3), a(e)))

    def energy(self, t1, t2):
        e = np.zeros(1)
        _check(load().ascc_energy(self._h, _ptr(np.ascontiguousarray(t1, np.float64)),
                                  _ptr(np.ascontiguousarray(t2, np.float64)), _ptr(e)))
        return float(e[0])

    def solve(self, check=False) -> Result:
        res = Result()
        st = load().ascc_solve(self._h, C.byref(res))
        if check:
            _check(st)
        elif st not in (0, 4, 5):
            _check(st)
        return res

    def solve_two_ansatz(self) -> TwoAnsatzResult:
        """Both ansatz choices of Sec. II.D and the reported energy (ascc_solve_two_ansatz)."""
        res = TwoAnsatzResult()
        st = load().ascc_solve_two_ansatz(self._h, C.byref(res))
        if st not in (0, 4, 5):
            _check(st)
        return res

    def checkpoint(self) -> bytes:
        """The iteration state (amplitudes, DIIS history, counters) as a host blob."""
        n = C.c_int64()
        _check(load().ascc_checkpoint_size(self._h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(load().ascc_checkpoint_save(self._h, buf, n.value))
        return buf.raw

    def restore(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(load().ascc_checkpoint_load(self._h, buf, len(blob)))

    def reset(self):
        _check(load().ascc_reset(self._h))

    def iterate(self, max_steps) -> Result:
        res = Result()
        st = load().ascc_iterate(self._h, int(max_steps), C.byref(res))
        if st not in (0, 4, 5):
            _check(st)
        return res

    def set_profiling(self, on=True):
        _check(load().ascc_set_profiling(self._h, int(bool(on))))

    def profile(self) -> Profile:
        p = Profile()
        _check(load().ascc_get_profile(self._h, C.byref(p)))
        return p

    def get_state(self):
        o, v = self.o, self.v
        t1 = np.zeros((o, v)); t2 = np.zeros((o, o, v, v)); t3 = np.zeros(self.n_t3)
        _check(load().ascc_get_state(self._h, _ptr(t1), _ptr(t2), _ptr(t3) if self.n_t3 else None))
        return t1, t2, t3

    def set_state(self, t1, t2, t3=None):
        t3 = None if t3 is None or self.n_t3 == 0 else np.ascontiguousarray(t3, np.float64)
        _check(load().ascc_set_state(self._h, _ptr(np.ascontiguousarray(t1, np.float64)),
                                     _ptr(np.ascontiguousarray(t2, np.float64)), _ptr(t3)))

    def launches(self) -> int:
        return int(load().ascc_launch_count(self._h))


class Server:
    """Continuous-batching request server (ascc_server_*): queue solves, drain, read results."""

    def __init__(self, memory_budget, max_active=4, options=None, **opt_kw):
        opt = options if options is not None else default_options()
        for k, val in opt_kw.items():
            setattr(opt, k, val)
        h = C.c_void_p()
        _check(load().ascc_server_create(C.byref(h), int(memory_budget), int(max_active),
                                         C.byref(opt)))
        self._h = h

    def submit(self, o, v, naux, eps, B, states):
        """states: list of (hole, particle) or None (ground state)."""
        eps = np.ascontiguousarray(eps, np.float64)
        B = np.ascontiguousarray(B, np.float64)
        arr = (Excitation * len(states))()
        for k, st in enumerate(states):
            arr[k] = (Excitation(0, 0, 0, 0.0, 0.0, 0, 0) if st is None
                      else Excitation(1, st[0], st[1], 0.0, 0.0, 0, 0))
        rid = C.c_int64()
        _check(load().ascc_server_submit(self._h, o, v, naux, _ptr(eps), _ptr(B), len(states),
                                         arr, C.byref(rid)))
        return rid.value

    def drain(self):
        _check(load().ascc_server_drain(self._h))

    def results(self):
        n = int(load().ascc_server_result_count(self._h))
        buf = (ServeResult * max(n, 1))()
        _check(load().ascc_server_results(self._h, buf, n))
        return [dict(request_id=r.request_id, state_index=r.state_index, status=r.status,
                     energy=r.energy, iterations=r.iterations, worker=r.worker,
                     t_arrival=r.t_arrival, t_start=r.t_start, t_end=r.t_end)
                for r in buf[:n]]

    def close(self):
        if getattr(self, "_h", None):
            load().ascc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
