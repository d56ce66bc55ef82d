"""The C-ABI library builds, loads and exports what include/rtt.h declares;
argument errors are reported without touching a GPU (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2604_22718_gb300 import build as rtt_build
from paper_2604_22718_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    rtt_build.build()
    from paper_2604_22718_gb300 import rtt
    return rtt.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(rtt_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"rtt_create", "rtt_destroy", "rtt_log_amplitudes", "rtt_local_energy",
            "rtt_mcmc_sweep", "rtt_observables"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_status_strings(lib):
    lib.rtt_status_string.restype = ctypes.c_char_p
    assert lib.rtt_status_string(0) == b"RTT_OK"
    assert lib.rtt_status_string(6) == b"RTT_ERR_UNSUPPORTED"


def _desc(inst, **kw):
    from paper_2604_22718_gb300 import rtt
    keep = dict(path=np.ascontiguousarray(inst.path, np.int32),
                t=np.ascontiguousarray(inst.tensors), bl=np.ascontiguousarray(inst.b_left),
                br=np.ascontiguousarray(inst.b_right),
                bonds=np.ascontiguousarray(inst.bonds, np.int32))
    keep.update(kw)
    d = rtt._Desc(inst.n_spins, keep["path"].shape[0], keep["t"].shape[2], keep["bonds"].shape[0],
                  keep["path"].ctypes.data, keep["t"].ctypes.data, keep["bl"].ctypes.data,
                  keep["br"].ctypes.data, keep["bonds"].ctypes.data, 1.0, 3.0,
                  kw.get("precision", 0), -1, 1)
    return d, keep


@pytest.mark.parametrize("mutate,expect", [
    ("path_out_of_range", 1),
    ("tc_bad_chi", 6),
    ("not_permutation", 6),
    ("nan_tensor", 4),
    ("bad_precision", 1),
    ("self_bond", 1),
])
def test_create_rejects_bad_descriptions_before_any_cuda_call(lib, mutate, expect):
    inst = inputs.make_instance(3, 3, 2, 4, 3.0, seed=1, mixing=False)
    path = inst.path.copy()
    t = inst.tensors.copy()
    bonds = inst.bonds.copy()
    prec = 0
    if mutate == "path_out_of_range":
        path[3] = 9
    elif mutate == "tc_bad_chi":            # FP16X3 needs chi in {64, 128}
        path[10], path[11] = path[11], path[10]   # (a general path is accepted)
        prec = 3
    elif mutate == "not_permutation":
        path[1] = path[0]
        path[10] = path[9]
    elif mutate == "nan_tensor":
        t[2, 1, 0, 0] = np.nan
    elif mutate == "bad_precision":
        prec = 7
    elif mutate == "self_bond":
        bonds[0, 1] = bonds[0, 0]
    d, keep = _desc(inst, path=path, t=t, bonds=bonds, precision=prec)
    h = ctypes.c_void_p()
    st = lib.rtt_create(ctypes.byref(d), ctypes.byref(h))
    assert st == expect
    assert h.value is None
    lib.rtt_last_error.restype = ctypes.c_char_p
    assert lib.rtt_last_error().startswith(b"rtt_create")
    if mutate == "tc_bad_chi":
        assert b"chi" in lib.rtt_last_error()


def test_null_handle_is_an_argument_error(lib):
    assert lib.rtt_log_amplitudes(None, None, 4, None, None, None, None) == 1
    assert lib.rtt_local_energy(None, None, 4, None, None, None) == 1
    assert lib.rtt_mcmc_sweep(None, None, None, 4, 0, 0, 1, 1, None, None, None) == 1
    assert lib.rtt_reserve(None, 4) == 1


def test_uniforms_empty_request_needs_no_gpu(lib):
    assert lib.rtt_mcmc_uniforms(1, 0, None, None, None) == 0
    assert lib.rtt_mcmc_uniforms(1, -1, None, None, None) == 1


def test_replica_plan_calls_reject_bad_arguments_before_any_cuda_call(lib):
    """rtt_tt_plan_create validates sizes, ranks, precision and string codes
    before it selects a device; the plan calls reject a null plan."""
    P = ctypes.c_void_p
    ops = np.zeros((2, 8), dtype=np.uint8)
    eta = np.ones(2)
    out = P()

    def create(length=8, chi=2, chi_tree=0, precision=0, n_terms=2, o=ops):
        return lib.rtt_tt_plan_create(ctypes.c_int32(length), ctypes.c_int32(chi),
                                      ctypes.c_int32(chi_tree), ctypes.c_int32(precision),
                                      ctypes.c_int32(n_terms), o.ctypes.data_as(P),
                                      eta.ctypes.data_as(P), ctypes.c_int32(0), ctypes.byref(out))
    assert create(length=1) == 1                         # RTT_ERR_INVALID_ARG
    assert create(n_terms=0) == 1
    assert create(chi=17) == 6                           # RTT_ERR_UNSUPPORTED
    assert create(precision=2) == 6                      # only FP64 and FP32
    assert create(chi=4, chi_tree=3) == 1                # chi <= chi_tree <= 16
    assert create(chi_tree=17) == 1
    bad = ops.copy()
    bad[1, 3] = 3                                        # string codes are 0, 1, 2
    assert create(o=bad) == 1
    assert out.value is None
    assert lib.rtt_tt_power(None, None, 0.1, 1, None, None) == 1
    assert lib.rtt_tt_apply(None, None, 0, None, None, None) == 1
    assert lib.rtt_tt_sum_round(None, 1, None, 0, None, None, None, None) == 1
    assert lib.rtt_tt_plan_destroy(None) == 0


def test_made_and_batch_calls_reject_bad_arguments_before_any_cuda_call(lib):
    """The learned-proposal and batched entry points: null handles, a
    non-permutation order and missing inputs are argument errors that
    need no GPU; destroying a null handle is a no-op."""
    P = ctypes.c_void_p
    out = P()
    order = np.array([0, 1, 1, 3], dtype=np.int32)           # not a permutation
    w = np.zeros(1000)
    assert lib.rtt_made_create(4, 8, order.ctypes.data, w.ctypes.data, 1, 0, ctypes.byref(out)) == 1
    good = np.arange(4, dtype=np.int32)
    assert lib.rtt_made_create(0, 8, good.ctypes.data, w.ctypes.data, 1, 0, ctypes.byref(out)) == 1
    assert lib.rtt_made_create(4, 8, good.ctypes.data, None, 1, 0, ctypes.byref(out)) == 1
    assert out.value is None
    assert lib.rtt_made_log_prob(None, None, 4, None, None) == 1
    assert lib.rtt_made_sample(None, 4, 0, 0, None, None, None) == 1
    assert lib.rtt_made_train_step(None, None, 4, 1e-3, None, None) == 1
    assert lib.rtt_made_set_inference(None, 1) == 1
    assert lib.rtt_made_set_training(None, 1) == 1
    assert lib.rtt_indep_mh(None, None, None, None, 4, 0, 0, None, None) == 1
    assert lib.rtt_made_destroy(None) == 0
    chains = np.array([16], dtype=np.int64)
    assert lib.rtt_batch_create(None, 1, chains.ctypes.data, ctypes.byref(out)) == 1
    assert lib.rtt_batch_step(None, None, None, 0, None, None, 0, None) == 1
    assert lib.rtt_batch_layout(None, None, None, None, None) == 1
    assert lib.rtt_batch_destroy(None) == 0


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 1000, 4097, 1 << 20])
def test_training_row_order_is_a_permutation(lib, n):
    """rtt_made_permutation (host only): every row of [0, n) exactly once, a
    different order for another pass or another seed."""
    from paper_2604_22718_gb300 import rtt
    p0 = rtt.made_permutation(n, 7, 0)
    assert np.array_equal(np.sort(p0), np.arange(n))
    if n >= 64:
        p1 = rtt.made_permutation(n, 7, 1)
        q0 = rtt.made_permutation(n, 8, 0)
        assert np.array_equal(np.sort(p1), np.arange(n))
        assert not np.array_equal(p0, p1) and not np.array_equal(p0, q0)
        # not close to the identity: few fixed points, rows spread over the range
        assert np.mean(p0 == np.arange(n)) < 0.05
        assert abs(np.corrcoef(p0, np.arange(n))[0, 1]) < 0.2


def test_training_loop_rejects_bad_arguments(lib):
    from paper_2604_22718_gb300 import rtt
    dummy = ctypes.c_void_p(1)        # never dereferenced: the checks come first
    data = ctypes.c_void_p(2)
    f = lib.rtt_made_fit
    assert f(None, data, 10, 1, 5, ctypes.c_float(1e-3), 0, None, None) == 1
    assert f(dummy, None, 10, 1, 5, ctypes.c_float(1e-3), 0, None, None) == 1
    assert f(dummy, data, 10, 1, 11, ctypes.c_float(1e-3), 0, None, None) == 1     # batch > n
    assert f(dummy, data, 10, 1, 0, ctypes.c_float(1e-3), 0, None, None) == 1
    assert f(dummy, data, 10, -1, 5, ctypes.c_float(1e-3), 0, None, None) == 1
    assert f(dummy, data, 10, 1, 5, ctypes.c_float(0.0), 0, None, None) == 1
    out = np.zeros(3, dtype=np.int64)
    assert lib.rtt_made_permutation(0, 1, 0, out.ctypes.data) == 1
    with pytest.raises(rtt.RTTError, match="INVALID_ARG"):
        rtt.made_permutation(0, 1, 0)


def test_wait_selftest_rejects_a_null_handle(lib):
    assert lib.rtt_wait_selftest(None, 2000000, None) == 1


def test_noalloc_energy_rejects_a_null_handle(lib):
    e = np.zeros(4)
    assert lib.rtt_local_energy_noalloc(None, None, 4, e.ctypes.data, None, None) == 1
    assert np.all(e == 0)
