"""Thin ctypes binding of librtt.so (include/rtt.h).

Argument marshalling only: every step of the sampler runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current CUDA stream.
If librtt.so is missing this module raises at import of the library -- there
is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librtt.so")

RTT_FP64, RTT_FP32, RTT_BF16X3, RTT_FP16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": RTT_FP64, "fp32": RTT_FP32, "bf16x3": RTT_BF16X3, "fp16x3": RTT_FP16X3}
STATUS = {0: "RTT_OK", 1: "RTT_ERR_INVALID_ARG", 2: "RTT_ERR_CUDA", 3: "RTT_ERR_OOM",
          4: "RTT_ERR_NUMERIC", 5: "RTT_ERR_TIMEOUT", 6: "RTT_ERR_UNSUPPORTED"}


class RTTError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("n_spins", ctypes.c_int32), ("length", ctypes.c_int32),
                ("chi", ctypes.c_int32), ("n_bonds", ctypes.c_int32),
                ("path", ctypes.c_void_p), ("tensors", ctypes.c_void_p),
                ("b_left", ctypes.c_void_p), ("b_right", ctypes.c_void_p),
                ("bonds", ctypes.c_void_p), ("J", ctypes.c_double), ("h", ctypes.c_double),
                ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class _KTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("var", ctypes.c_double), ("se", ctypes.c_double),
                ("se_bin", ctypes.c_double), ("se_chain", ctypes.c_double),
                ("tau_int", ctypes.c_double), ("ess", ctypes.c_double),
                ("v_score", ctypes.c_double), ("accept_rate", ctypes.c_double),
                ("n", ctypes.c_int64), ("window", ctypes.c_int32), ("pad", ctypes.c_int32)]


_lib = None


def lib():
    """Load librtt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2604_22718_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        L.rtt_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(P)]
        L.rtt_destroy.argtypes = [P]
        L.rtt_reserve.argtypes = [P, I64]
        L.rtt_scratch_bytes.argtypes = [P, I64, ctypes.POINTER(ctypes.c_size_t)]
        L.rtt_log_amplitudes.argtypes = [P, P, I64, P, P, P, P]
        L.rtt_local_energy.argtypes = [P, P, I64, P, P, P]
        L.rtt_mixed_local_energy.argtypes = [P, P, P, I64, P, P, P]
        L.rtt_create_sum.argtypes = [ctypes.POINTER(_Desc), I32, P, ctypes.POINTER(P)]
        L.rtt_dual_solve.argtypes = [I32, P, P, P, P, P]
        L.rtt_dual_gram_schmidt.argtypes = [I32, P, I32, P]
        L.rtt_dual_back_transform.argtypes = [I32, P, P, P]
        L.rtt_dual_step.argtypes = [P, I32, P, P, I64, I64, I64, P, P, P, P]
        L.rtt_mcmc_sweep.argtypes = [P, P, P, I64, I64, I64, I32, I32, P, P, P]
        L.rtt_observables.argtypes = [P, P, I32, I64, P, I64, ctypes.POINTER(_Stats), P]
        L.rtt_mcmc_uniforms.argtypes = [U64, I64, P, P, P]
        L.rtt_wait_selftest.argtypes = [P, I64, P]
        L.rtt_device_status.argtypes = [P, ctypes.POINTER(I32)]
        L.rtt_profile.argtypes = [P, I32]
        L.rtt_profile_read.argtypes = [P, ctypes.POINTER(_KTime), I32, ctypes.POINTER(I32)]
        L.rtt_batch_create.argtypes = [P, I32, P, ctypes.POINTER(P)]
        L.rtt_batch_destroy.argtypes = [P]
        L.rtt_batch_layout.argtypes = [P, P, P, P, P]
        L.rtt_batch_init.argtypes = [P, P, P, P]
        L.rtt_batch_step.argtypes = [P, P, P, I64, P, P, I32, P]
        L.rtt_batch_tune.argtypes = [P, ctypes.c_char_p, I32, P]
        L.rtt_batch_shape.argtypes = [P, I32, P, P]
        for name in ("rtt_batch_create", "rtt_batch_destroy", "rtt_batch_layout", "rtt_batch_init",
                     "rtt_batch_step", "rtt_batch_tune", "rtt_batch_shape"):
            getattr(L, name).restype = ctypes.c_int
        L.rtt_made_create.argtypes = [I32, I32, P, P, U64, I32, ctypes.POINTER(P)]
        L.rtt_made_destroy.argtypes = [P]
        L.rtt_made_get_params.argtypes = [P, P]
        L.rtt_made_gradients.argtypes = [P, P, I64, P, P, P]
        L.rtt_made_train_step.argtypes = [P, P, I64, ctypes.c_float, P, P]
        L.rtt_made_log_prob.argtypes = [P, P, I64, P, P]
        L.rtt_made_sample.argtypes = [P, I64, I64, I64, P, P, P]
        L.rtt_indep_mh.argtypes = [P, P, P, P, I64, I64, I64, P, P]
        L.rtt_made_fit.argtypes = [P, P, I64, I32, I32, ctypes.c_float, U64, P, P]
        L.rtt_made_permutation.argtypes = [I64, U64, I64, P]
        L.rtt_made_set_training.argtypes = [P, I32]
        L.rtt_made_set_training.restype = ctypes.c_int
        L.rtt_made_set_inference.argtypes = [P, I32]
        L.rtt_made_device_status.argtypes = [P, ctypes.POINTER(I32)]
        L.rtt_made_set_inference.restype = ctypes.c_int
        L.rtt_made_device_status.restype = ctypes.c_int
        for name in ("rtt_made_create", "rtt_made_destroy", "rtt_made_get_params",
                     "rtt_made_gradients", "rtt_made_train_step", "rtt_made_log_prob",
                     "rtt_made_sample", "rtt_indep_mh", "rtt_made_fit", "rtt_made_permutation"):
            getattr(L, name).restype = ctypes.c_int
        L.rtt_replica_lift.argtypes = [I32, I32, P, I32, P, P, P, P, P, P, P]
        L.rtt_tt_plan_create.argtypes = [I32, I32, I32, I32, I32, P, P, I32, ctypes.POINTER(P)]
        L.rtt_tt_plan_destroy.argtypes = [P]
        L.rtt_tt_power.argtypes = [P, P, ctypes.c_double, I32, P, P]
        L.rtt_tt_round_sum.argtypes = [P, P, P, ctypes.c_double, P, P, ctypes.c_double, P, P, P]
        L.rtt_tt_apply.argtypes = [P, P, I32, P, P, P]
        L.rtt_tt_sum_round.argtypes = [P, I32, P, I32, P, P, P, P]
        for name in ("rtt_replica_lift", "rtt_tt_plan_create", "rtt_tt_plan_destroy",
                     "rtt_tt_power", "rtt_tt_round_sum", "rtt_tt_apply", "rtt_tt_sum_round"):
            getattr(L, name).restype = ctypes.c_int
        L.rtt_status_string.argtypes = [I32]
        L.rtt_status_string.restype = ctypes.c_char_p
        L.rtt_last_error.restype = ctypes.c_char_p
        for name in ("rtt_create", "rtt_destroy", "rtt_reserve", "rtt_scratch_bytes",
                     "rtt_log_amplitudes", "rtt_local_energy", "rtt_mcmc_sweep",
                     "rtt_observables", "rtt_mcmc_uniforms", "rtt_profile", "rtt_profile_read",
                     "rtt_wait_selftest", "rtt_device_status"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _desc_of(inst, precision: int, device: int, seed: int):
    """rtt_desc of an instance and the host arrays it points into (keep them alive)."""
    path = np.ascontiguousarray(inst.path, dtype=np.int32)
    t = np.ascontiguousarray(inst.tensors, dtype=np.float64)
    bl = np.ascontiguousarray(inst.b_left, dtype=np.float64)
    br = np.ascontiguousarray(inst.b_right, dtype=np.float64)
    bonds = np.ascontiguousarray(inst.bonds, dtype=np.int32).reshape(-1, 2)
    L, _, chi, _ = t.shape
    d = _Desc(int(inst.n_spins), L, chi, bonds.shape[0], path.ctypes.data, t.ctypes.data,
              bl.ctypes.data, br.ctypes.data, bonds.ctypes.data if bonds.size else None,
              float(inst.J), float(inst.h), precision, device, int(seed))
    return d, (path, t, bl, br, bonds)


def dual_solve(Ht, St):
    """rtt_dual_solve: eigenvalues of H~ c = lambda S~ c (complex, by increasing
    real part) and the scaled eigenvector of the lowest one (NaN if not real)."""
    Ht = np.ascontiguousarray(Ht, dtype=np.float64)
    St = np.ascontiguousarray(St, dtype=np.float64)
    M = Ht.shape[0]
    assert Ht.shape == (M, M) and St.shape == (M, M)
    re, im, c = np.empty(M), np.empty(M), np.empty(M)
    _check(lib().rtt_dual_solve(M, Ht.ctypes.data, St.ctypes.data, re.ctypes.data, im.ctypes.data,
                                c.ctypes.data), "rtt_dual_solve")
    return re + 1j * im, c


def dual_gram_schmidt(St, first_only: bool):
    """rtt_dual_gram_schmidt: T with psi' = T psi (Eq. Gram-Schmid)."""
    St = np.ascontiguousarray(St, dtype=np.float64)
    M = St.shape[0]
    assert St.shape == (M, M)
    T = np.empty((M, M))
    _check(lib().rtt_dual_gram_schmidt(M, St.ctypes.data, int(bool(first_only)), T.ctypes.data),
           "rtt_dual_gram_schmidt")
    return T


def dual_back_transform(T, c_prime):
    """rtt_dual_back_transform: c = T^T c' on the original states."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    cp = np.ascontiguousarray(c_prime, dtype=np.float64)
    M = cp.shape[0]
    assert T.shape == (M, M)
    c = np.empty(M)
    _check(lib().rtt_dual_back_transform(M, T.ctypes.data, cp.ctypes.data, c.ctypes.data),
           "rtt_dual_back_transform")
    return c


def dual_step(handles, spins, states, sweep: int, e_mixed=None, ratio=None, n_accept=None,
              chain0: int = 0, stream=None):
    """rtt_dual_step for M RTT objects: spins/states/n_accept lists of device
    tensors [B][N] uint8, [B][2] int64, [B] int64; e_mixed, ratio [M][M][B] float64."""
    M = len(handles)
    B = spins[0].shape[0]
    for m in range(M):
        _dev_check(spins[m], torch.uint8, (B, handles[m].n), "spins")
        _dev_check(states[m], torch.int64, (B, 2), "state")
    for t, nm in ((e_mixed, "e_mixed"), (ratio, "ratio")):
        if t is not None:
            _dev_check(t, torch.float64, (M, M, B), nm)
    H = (ctypes.c_void_p * M)(*[h._h.value for h in handles])
    S = (ctypes.c_void_p * M)(*[_ptr(x).value for x in spins])
    T = (ctypes.c_void_p * M)(*[_ptr(x).value for x in states])
    A = (ctypes.c_void_p * M)(*[(_ptr(x).value if x is not None else None)
                                for x in (n_accept or [None] * M)])
    _check(lib().rtt_dual_step(H, M, S, T, B, int(chain0), int(sweep), _ptr(e_mixed), _ptr(ratio),
                               A if n_accept is not None else None, _stream(stream)),
           "rtt_dual_step")


def _check(status: int, where: str):
    if status != 0:
        raise RTTError(status, where, lib().rtt_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_check(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def new_state(B: int, device="cuda") -> torch.Tensor:
    """Chain-state buffer: int64 [B, 2] holding (mant as float64 bits, exp2)."""
    return torch.zeros((B, 2), dtype=torch.int64, device=device)


def state_mant(state: torch.Tensor) -> torch.Tensor:
    return state.view(torch.float64)[:, 0]


def state_exp(state: torch.Tensor) -> torch.Tensor:
    return state[:, 1]


class RTT:
    """One RTT instance on one GPU (wraps an rtt_handle)."""

    def __init__(self, inst, precision: str | int = "fp32", device: int | None = None,
                 seed: int = 22718):
        self.inst = inst
        self.n = int(inst.n_spins) if inst is not None else 0
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.seed = int(seed)
        if inst is None:            # filled by from_sum
            self._h = None
            return
        d, self._keep = _desc_of(inst, self.precision, self.device, self.seed)
        self.L, self.chi = int(d.length), int(d.chi)
        h = ctypes.c_void_p()
        _check(lib().rtt_create(ctypes.byref(d), ctypes.byref(h)), "rtt_create")
        self._h = h

    @classmethod
    def from_sum(cls, instances, coef, precision: str | int = "fp32", device: int | None = None,
                 seed: int = 22718):
        """One RTT for sum_m coef[m] psi^m (rtt_create_sum: block-diagonal direct sum)."""
        self = cls(None, precision, device, seed)
        M = len(instances)
        descs = (_Desc * M)()
        keep = []
        for m, inst in enumerate(instances):
            d, k = _desc_of(inst, self.precision, self.device, self.seed)
            descs[m] = d
            keep.append(k)
        c = np.ascontiguousarray(coef, dtype=np.float64)
        assert c.shape == (M,)
        h = ctypes.c_void_p()
        _check(lib().rtt_create_sum(descs, M, c.ctypes.data, ctypes.byref(h)), "rtt_create_sum")
        self._h = h
        self.n = int(instances[0].n_spins)
        self.L = int(np.asarray(instances[0].path).shape[0])
        self.chi = int(sum(int(i.tensors.shape[2]) for i in instances))
        self.inst = None
        return self

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rtt_destroy(self._h)
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

    @property
    def handle(self):
        return self._h

    def reserve(self, B: int):
        _check(lib().rtt_reserve(self._h, int(B)), "rtt_reserve")

    def scratch_bytes(self, B: int) -> int:
        out = ctypes.c_size_t()
        _check(lib().rtt_scratch_bytes(self._h, int(B), ctypes.byref(out)), "rtt_scratch_bytes")
        return int(out.value)

    def profile(self, enable: bool = True):
        _check(lib().rtt_profile(self._h, 1 if enable else 0), "rtt_profile")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} since the last read (synchronises)."""
        buf = (_KTime * 32)()
        n = ctypes.c_int32()
        _check(lib().rtt_profile_read(self._h, buf, 32, ctypes.byref(n)), "rtt_profile_read")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms))
                for i in range(min(n.value, 32))}

    def device_status(self):
        """(status, flags) of rtt_device_status: the handle's device error flags
        since the last call (bit 0: a bounded wait ran out), then cleared."""
        f = ctypes.c_int32()
        st = lib().rtt_device_status(self._h, ctypes.byref(f))
        return int(st), int(f.value)

    def wait_selftest(self, budget_cycles: int, stream=None):
        """rtt_wait_selftest: one bounded wait that nothing completes."""
        _check(lib().rtt_wait_selftest(self._h, int(budget_cycles), _stream(stream)),
               "rtt_wait_selftest")

    def log_amplitudes(self, spins: torch.Tensor, stream=None):
        B = spins.shape[0]
        _dev_check(spins, torch.uint8, (B, self.n), "spins")
        la = torch.empty(B, dtype=torch.float64, device=spins.device)
        sg = torch.empty(B, dtype=torch.int8, device=spins.device)
        st = new_state(B, spins.device)
        _check(lib().rtt_log_amplitudes(self._h, _ptr(spins), B, _ptr(la), _ptr(sg), _ptr(st),
                                        _stream(stream)), "rtt_log_amplitudes")
        return la, sg, st

    def local_energy(self, spins: torch.Tensor, with_ratios: bool = False, stream=None):
        B = spins.shape[0]
        _dev_check(spins, torch.uint8, (B, self.n), "spins")
        e = torch.empty(B, dtype=torch.float64, device=spins.device)
        r = torch.empty((B, self.n), dtype=torch.float64, device=spins.device) if with_ratios else None
        _check(lib().rtt_local_energy(self._h, _ptr(spins), B, _ptr(e), _ptr(r), _stream(stream)),
               "rtt_local_energy")
        return (e, r) if with_ratios else e

    def mixed_local_energy(self, other: "RTT", spins: torch.Tensor, stream=None):
        """(E^{ab}(s), psi^b(s)/psi^a(s)) with a = self, b = other (dual Monte Carlo)."""
        B = spins.shape[0]
        _dev_check(spins, torch.uint8, (B, self.n), "spins")
        e = torch.empty(B, dtype=torch.float64, device=spins.device)
        r = torch.empty(B, dtype=torch.float64, device=spins.device)
        _check(lib().rtt_mixed_local_energy(self._h, other._h, _ptr(spins), B, _ptr(e), _ptr(r),
                                            _stream(stream)), "rtt_mixed_local_energy")
        return e, r

    def mcmc_sweep(self, spins: torch.Tensor, state: torch.Tensor, sweep0: int, n_sweeps: int,
                   measure_every: int = 1, trace: torch.Tensor | None = None,
                   n_accept: torch.Tensor | None = None, chain0: int = 0, stream=None):
        B = spins.shape[0]
        _dev_check(spins, torch.uint8, (B, self.n), "spins")
        _dev_check(state, torch.int64, (B, 2), "state")
        if trace is not None:
            rows = n_sweeps // measure_every if measure_every >= 1 else None
            _dev_check(trace, torch.float64, None if rows is None else (rows, B), "trace")
        if n_accept is not None:
            _dev_check(n_accept, torch.int64, (B,), "n_accept")
        _check(lib().rtt_mcmc_sweep(self._h, _ptr(spins), _ptr(state), B, int(chain0), int(sweep0),
                                    int(n_sweeps), int(measure_every), _ptr(trace), _ptr(n_accept),
                                    _stream(stream)), "rtt_mcmc_sweep")

    def observables(self, trace: torch.Tensor, n_accept: torch.Tensor | None = None,
                    proposals_per_chain: int = 0, stream=None) -> dict:
        T, B = trace.shape
        _dev_check(trace, torch.float64, (T, B), "trace")
        out = _Stats()
        _check(lib().rtt_observables(self._h, _ptr(trace), T, B, _ptr(n_accept),
                                     int(proposals_per_chain), ctypes.byref(out), _stream(stream)),
               "rtt_observables")
        return {k: getattr(out, k) for k, _ in _Stats._fields_ if k != "pad"}


def mcmc_uniforms(seed: int, counters: torch.Tensor, stream=None) -> torch.Tensor:
    """Device Philox uniforms for counters int64/uint64 [n][3] (chain, sweep, proposal)."""
    n = counters.shape[0]
    if counters.dtype not in (torch.int64, torch.uint64) or tuple(counters.shape) != (n, 3):
        raise ValueError("counters must be int64 [n][3]")
    out = torch.empty(n, dtype=torch.float64, device=counters.device)
    _check(lib().rtt_mcmc_uniforms(int(seed), n, _ptr(counters.contiguous()), _ptr(out),
                                   _stream(stream)), "rtt_mcmc_uniforms")
    return out


class RTTBatch:
    """Many RTT instances sampled together: FP32 ones by one persistent kernel
    per iteration, FP16X3 / BF16X3 ones (chi 64 or 128) on the tensor cores.
    precisions: one name per instance ("fp32", "fp16x3", "bf16x3"), default FP32."""

    def __init__(self, instances, chains, device: int | None = None, seeds=None, precisions=None):
        n = len(instances)
        chains = [int(c) for c in (chains if hasattr(chains, "__len__") else [chains] * n)]
        self.instances = list(instances)
        self.n = n
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._keep = []
        descs = (_Desc * n)()
        for i, inst in enumerate(instances):
            path = np.ascontiguousarray(inst.path, dtype=np.int32)
            t = np.ascontiguousarray(inst.tensors, dtype=np.float64)
            bl = np.ascontiguousarray(inst.b_left, dtype=np.float64)
            br = np.ascontiguousarray(inst.b_right, dtype=np.float64)
            bonds = np.ascontiguousarray(inst.bonds, dtype=np.int32).reshape(-1, 2)
            self._keep += [path, t, bl, br, bonds]
            seed = int(seeds[i]) if seeds is not None else 22722 + i
            descs[i] = _Desc(int(inst.n_spins), t.shape[0], t.shape[2], bonds.shape[0],
                             path.ctypes.data, t.ctypes.data, bl.ctypes.data, br.ctypes.data,
                             bonds.ctypes.data if bonds.size else None, float(inst.J),
                             float(inst.h), PRECISIONS[precisions[i]] if precisions else RTT_FP32,
                             self.device, seed)
        self._chains = np.asarray(chains, dtype=np.int64)
        b = ctypes.c_void_p()
        _check(lib().rtt_batch_create(descs, n, self._chains.ctypes.data, ctypes.byref(b)),
               "rtt_batch_create")
        self._b = b
        tc, ts = ctypes.c_int64(), ctypes.c_int64()
        self.chain_off = np.zeros(n, dtype=np.int64)
        self.spin_off = np.zeros(n, dtype=np.int64)
        _check(lib().rtt_batch_layout(b, ctypes.byref(tc), ctypes.byref(ts),
                                      self.chain_off.ctypes.data, self.spin_off.ctypes.data),
               "rtt_batch_layout")
        self.total_chains, self.total_spins = tc.value, ts.value
        self.chains = chains

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            lib().rtt_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init(self, spins: torch.Tensor, stream=None) -> torch.Tensor:
        _dev_check(spins, torch.uint8, (self.total_spins,), "spins")
        st = new_state(self.total_chains, spins.device)
        _check(lib().rtt_batch_init(self._b, _ptr(spins), _ptr(st), _stream(stream)), "rtt_batch_init")
        return st

    def step(self, spins, state, sweep: int, e_loc, n_accept=None, use_graph=True, stream=None):
        _dev_check(spins, torch.uint8, (self.total_spins,), "spins")
        _dev_check(state, torch.int64, (self.total_chains, 2), "state")
        _dev_check(e_loc, torch.float64, (self.total_chains,), "e_loc")
        if n_accept is not None:
            _dev_check(n_accept, torch.int64, (self.total_chains,), "n_accept")
        _check(lib().rtt_batch_step(self._b, _ptr(spins), _ptr(state), int(sweep), _ptr(e_loc),
                                    _ptr(n_accept), 1 if use_graph else 0, _stream(stream)),
               "rtt_batch_step")

    def tune(self, cache_path: str | None = None, probe_chains: int = 64, stream=None):
        _check(lib().rtt_batch_tune(self._b, cache_path.encode() if cache_path else None,
                                    int(probe_chains), _stream(stream)), "rtt_batch_tune")

    def shape(self, i: int):
        g, c = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rtt_batch_shape(self._b, int(i), ctypes.byref(g), ctypes.byref(c)),
               "rtt_batch_shape")
        return g.value, c.value


class MADE:
    """Learned autoregressive proposal (masked MLP) trained and sampled on the GPU."""

    def __init__(self, n_spins: int, hidden: int, order, init_weights, seed: int = 22723,
                 device: int | None = None):
        self.n, self.hidden = int(n_spins), int(hidden)
        self.order = np.ascontiguousarray(order, dtype=np.int32)
        w = np.ascontiguousarray(init_weights, dtype=np.float64)
        N, H = self.n, self.hidden
        self.P = H * N + H + H * H + H + N * H + N
        if w.shape != (self.P,):
            raise ValueError(f"init_weights must have {self.P} entries")
        self.device = torch.cuda.current_device() if device is None else int(device)
        m = ctypes.c_void_p()
        _check(lib().rtt_made_create(N, H, self.order.ctypes.data, w.ctypes.data, int(seed),
                                     self.device, ctypes.byref(m)), "rtt_made_create")
        self._m = m
        self.seed = int(seed)

    def close(self):
        if getattr(self, "_m", None) is not None and self._m.value:
            lib().rtt_made_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._m

    def set_inference(self, bf16: bool):
        """Tensor-core BF16 (True) or FP32 (False) arithmetic for the H x H layer
        of sampling and evaluation (rtt_made_set_inference)."""
        _check(lib().rtt_made_set_inference(self._m, 1 if bf16 else 0), "rtt_made_set_inference")

    def set_training(self, tc: bool):
        """Tensor-core BF16 hi/lo (True) or FP32 CUDA-core (False, the default)
        arithmetic for the training GEMMs (rtt_made_set_training)."""
        _check(lib().rtt_made_set_training(self._m, 1 if tc else 0), "rtt_made_set_training")

    def device_status(self) -> int:
        """Error flags of the model's tensor-core kernels since the last call (0 = none)."""
        f = ctypes.c_int32()
        st = lib().rtt_made_device_status(self._m, ctypes.byref(f))
        if st not in (0, 5):
            _check(st, "rtt_made_device_status")
        return int(f.value)

    def params(self) -> np.ndarray:
        out = np.empty(self.P, dtype=np.float32)
        _check(lib().rtt_made_get_params(self._m, out.ctypes.data), "rtt_made_get_params")
        return out

    def gradients(self, spins, stream=None):
        B = spins.shape[0]
        _dev_check(spins, torch.uint8, (B, self.n), "spins")
        g = torch.empty(self.P, dtype=torch.float32, device=spins.device)
        nll = torch.empty(1, dtype=torch.float64, device=spins.device)
        _check(lib().rtt_made_gradients(self._m, _ptr(spins), B, _ptr(g), _ptr(nll), _stream(stream)),
               "rtt_made_gradients")
        return g, nll

    def train_step(self, spins, lr: float = 1e-3, nll=None, stream=None):
        B = spins.shape[0]
        _dev_check(spins, torch.uint8, (B, self.n), "spins")
        _check(lib().rtt_made_train_step(self._m, _ptr(spins), B, float(lr), _ptr(nll),
                                         _stream(stream)), "rtt_made_train_step")

    def log_prob(self, spins, stream=None):
        B = spins.shape[0]
        _dev_check(spins, torch.uint8, (B, self.n), "spins")
        out = torch.empty(B, dtype=torch.float64, device=spins.device)
        _check(lib().rtt_made_log_prob(self._m, _ptr(spins), B, _ptr(out), _stream(stream)),
               "rtt_made_log_prob")
        return out

    def sample(self, B: int, chain0: int = 0, round: int = 0, stream=None):
        sp = torch.empty((B, self.n), dtype=torch.uint8, device="cuda")
        lq = torch.empty(B, dtype=torch.float64, device="cuda")
        _check(lib().rtt_made_sample(self._m, int(B), int(chain0), int(round), _ptr(sp), _ptr(lq),
                                     _stream(stream)), "rtt_made_sample")
        return sp, lq

    def fit(self, data: torch.Tensor, epochs: int, batch: int = 1024, lr: float = 1e-3,
            seed: int = 0, stream=None):
        """rtt_made_fit: minibatch Adam over `data` (device uint8 [n][N]) in a
        keyed random row order per epoch; returns the mean NLL of each epoch."""
        n = data.shape[0]
        _dev_check(data, torch.uint8, (n, self.n), "data")
        hist = np.zeros(max(int(epochs), 0), dtype=np.float64)
        _check(lib().rtt_made_fit(self._m, _ptr(data), n, int(epochs), int(batch), float(lr),
                                  int(seed), hist.ctypes.data if hist.size else None,
                                  _stream(stream)), "rtt_made_fit")
        return [float(x) for x in hist]


def made_permutation(n: int, seed: int, epoch: int) -> np.ndarray:
    """rtt_made_permutation: the training loop's row order for one epoch."""
    out = np.empty(int(n), dtype=np.int64)
    _check(lib().rtt_made_permutation(int(n), int(seed), int(epoch), out.ctypes.data),
           "rtt_made_permutation")
    return out


def indep_mh(model: RTT, made: MADE, spins, state, round: int, n_accept=None, chain0: int = 0,
             stream=None):
    """One learned independence proposal per chain (in place)."""
    B = spins.shape[0]
    _dev_check(spins, torch.uint8, (B, model.n), "spins")
    _dev_check(state, torch.int64, (B, 2), "state")
    if n_accept is not None:
        _dev_check(n_accept, torch.int64, (B,), "n_accept")
    _check(lib().rtt_indep_mh(model.handle, made.handle, _ptr(spins), _ptr(state), B, int(chain0),
                              int(round), _ptr(n_accept), _stream(stream)), "rtt_indep_mh")


# ---------------------------------------------------------------- replica space

def replica_lift(n_spins: int, path, terms):
    """rtt_replica_lift: physical Pauli terms [(coef, [(spin, 'X'|'Z'), ...], block)]
    -> (eta [K] float64, ops [K][L] uint8 string codes: 0 I, 1 X, 2 Z)."""
    code = {"X": 1, "Z": 2, "Y": 3}
    path = np.ascontiguousarray(path, dtype=np.int32)
    L = path.shape[0]
    K = len(terms)
    coef = np.ascontiguousarray([t[0] for t in terms], dtype=np.float64)
    block = np.ascontiguousarray([t[2] for t in terms], dtype=np.int32)
    off = np.zeros(K + 1, dtype=np.int32)
    spins, ops = [], []
    for k, (_, factors, _) in enumerate(terms):
        for j, op in factors:
            spins.append(int(j))
            ops.append(code[op])
        off[k + 1] = len(spins)
    spins = np.ascontiguousarray(spins if spins else [0], dtype=np.int32)
    ops = np.ascontiguousarray(ops if ops else [0], dtype=np.uint8)
    out = np.zeros((max(K, 1), L), dtype=np.uint8)
    eta = np.zeros(max(K, 1), dtype=np.float64)
    _check(lib().rtt_replica_lift(int(n_spins), L, path.ctypes.data, K, coef.ctypes.data,
                                  block.ctypes.data, off.ctypes.data, spins.ctypes.data,
                                  ops.ctypes.data, out.ctypes.data, eta.ctypes.data),
           "rtt_replica_lift")
    return eta[:K], out[:K]


class TTPlan:
    """rtt_tt_plan: (1 - tau H-bar) steps and two-term roundings on TTs of
    `length` sites and rank chi; H-bar = sum_k eta[k] P_k (ops [K][length]);
    the tree's pairwise sums are rounded to chi_tree (0: 2 chi, at most 16)."""

    def __init__(self, length: int, chi: int, eta, ops, device: int = 0, precision: str = "fp64",
                 chi_tree: int = 0):
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        if ops.ndim != 2 or ops.shape != (eta.shape[0], length):
            raise ValueError("ops must have shape [len(eta)][length]")
        self.length, self.chi = int(length), int(chi)
        self._p = ctypes.c_void_p()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib().rtt_tt_plan_create(self.length, self.chi, int(chi_tree), prec, eta.shape[0],
                                        ops.ctypes.data, eta.ctypes.data, int(device),
                                        ctypes.byref(self._p)),
               "rtt_tt_plan_create")

    def close(self):
        if getattr(self, "_p", None) is not None and self._p.value:
            lib().rtt_tt_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cores(self, t, name):
        _dev_check(t, torch.float64, (self.length, 2, self.chi, self.chi), name)

    def power(self, phi: torch.Tensor, tau: float, steps: int, log_norm: torch.Tensor = None,
              stream=None):
        """phi (device float64 [L][2][chi][chi]) <- (1 - tau H-bar)^steps phi, each
        step rounded and scaled to unit norm; log_norm (device float64 [steps])."""
        self._cores(phi, "phi")
        if log_norm is not None:
            _dev_check(log_norm, torch.float64, (steps,), "log_norm")
        _check(lib().rtt_tt_power(self._p, _ptr(phi), float(tau), int(steps), _ptr(log_norm),
                                  _stream(stream)), "rtt_tt_power")

    def round_sum(self, a, b, out, coef_a: float = 1.0, coef_b: float = 1.0, ops_a=None,
                  ops_b=None, log_norm=None, stream=None):
        """out <- round(coef_a P_a a + coef_b P_b b); ops_* device uint8 [L] or None."""
        for t, nm in ((a, "a"), (b, "b"), (out, "out")):
            self._cores(t, nm)
        for t, nm in ((ops_a, "ops_a"), (ops_b, "ops_b")):
            if t is not None:
                _dev_check(t, torch.uint8, (self.length,), nm)
        if log_norm is not None:
            _dev_check(log_norm, torch.float64, (1,), "log_norm")
        _check(lib().rtt_tt_round_sum(self._p, _ptr(a), _ptr(ops_a), float(coef_a), _ptr(b),
                                      _ptr(ops_b), float(coef_b), _ptr(out), _ptr(log_norm),
                                      _stream(stream)), "rtt_tt_round_sum")

    def apply(self, phi: torch.Tensor, out: torch.Tensor, log_norm: torch.Tensor = None,
              stream=None):
        """out <- round(H-bar phi) / norm for the plan's operator (rtt_tt_apply);
        phi may have a smaller rank (padded cores [L][2][c][c]) than the plan's."""
        c = int(phi.shape[2]) if phi.dim() == 4 else 0
        _dev_check(phi, torch.float64, (self.length, 2, c, c), "phi")
        self._cores(out, "out")
        if log_norm is not None:
            _dev_check(log_norm, torch.float64, (1,), "log_norm")
        _check(lib().rtt_tt_apply(self._p, _ptr(phi), c, _ptr(out), _ptr(log_norm), _stream(stream)),
               "rtt_tt_apply")

    def sum_round(self, tts, coef, out: torch.Tensor, log_norm: torch.Tensor = None, stream=None):
        """out <- round(sum_m coef[m] tts[m]) / norm (rtt_tt_sum_round)."""
        c = int(tts[0].shape[2]) if tts and tts[0].dim() == 4 else 0
        for m, t in enumerate(tts):
            _dev_check(t, torch.float64, (self.length, 2, c, c), f"tts[{m}]")
        self._cores(out, "out")
        if log_norm is not None:
            _dev_check(log_norm, torch.float64, (1,), "log_norm")
        n = len(tts)
        c_in = c
        ptrs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in tts])
        cf = np.ascontiguousarray(coef, dtype=np.float64)
        if cf.shape != (n,):
            raise ValueError("coef must have one entry per TT")
        _check(lib().rtt_tt_sum_round(self._p, n, ptrs, c_in, cf.ctypes.data, _ptr(out),
                                      _ptr(log_norm), _stream(stream)), "rtt_tt_sum_round")
