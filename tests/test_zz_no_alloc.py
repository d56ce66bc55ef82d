"""rtt_local_energy_noalloc: the local energy from a call that allocates no
device memory, for callers that cannot allocate at that moment (loops that
forbid allocator calls after start-up, programs whose device memory belongs
to an external pool manager).  It must give the same results as
rtt_local_energy, call after call, while its scratch comes from the library's
fixed static device array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import pytest
import torch

from paper_2604_22718_gb300 import inputs

pytestmark = pytest.mark.gpu


def _noalloc():
    from paper_2604_22718_gb300 import build, rtt
    build.build()
    f = rtt.lib().rtt_local_energy_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return rtt, f


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    rtt, f = _noalloc()
    inst = inputs.workload("plain_6x6")
    B = 512
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with rtt.RTT(inst, prec) as m:
        for call in range(2):
            spins = torch.from_numpy(inputs.initial_spins(100 + call, B, inst.n_spins)).cuda()
            e_ref, r_ref = m.local_energy(spins, with_ratios=True)
            e = torch.empty(B, dtype=torch.float64, device="cuda")
            r = torch.empty((B, inst.n_spins), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            st = f(m.handle, _p(spins), B, _p(e), _p(r), stream)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            assert st == 0, rtt.lib().rtt_last_error()
            # identical kernels on identical inputs: bit-identical results
            assert torch.equal(e, e_ref)
            assert torch.equal(r, r_ref)
            if call == 1:   # the first call may load the library's device image
                assert abs(free_after - free_before) < 2 * 2**20


def test_noalloc_rejects_a_batch_beyond_the_static_area():
    rtt, f = _noalloc()
    inst = inputs.workload("plain_6x6")
    B = 8192    # ~19 KB of scratch per chain in FP32: needs > 32 MiB
    spins = torch.zeros((B, inst.n_spins), dtype=torch.uint8, device="cuda")
    e = torch.empty(B, dtype=torch.float64, device="cuda")
    with rtt.RTT(inst, "fp32") as m:
        st = f(m.handle, _p(spins), B, _p(e), None, None)
    assert st == 1
    assert b"static area" in rtt.lib().rtt_last_error()


def test_noalloc_rejects_a_batch_whose_size_would_overflow():
    """A batch so large that its scratch size overflows 64-bit arithmetic is
    rejected as too large before anything is launched."""
    rtt, f = _noalloc()
    inst = inputs.workload("plain_6x6")
    e = torch.full((4,), 3.5, dtype=torch.float64, device="cuda")
    spins = torch.zeros((4, inst.n_spins), dtype=torch.uint8, device="cuda")
    with rtt.RTT(inst, "fp32") as m:
        for B in (1 << 62, (1 << 63) - 1, 1 << 40):
            assert f(m.handle, _p(spins), B, _p(e), None, None) == 1
            assert b"static area" in rtt.lib().rtt_last_error()
    torch.cuda.synchronize()
    assert torch.all(e == 3.5)


def test_noalloc_rejects_unsupported_handles_and_null_arguments():
    """Split-precision handles and general paths are not served
    (RTT_ERR_UNSUPPORTED), null spins or e_loc are argument errors; in every
    case e_loc is left as it was."""
    rtt, f = _noalloc()
    B = 16
    e = torch.full((B,), -2.0, dtype=torch.float64, device="cuda")
    with rtt.RTT(inputs.make_instance(3, 3, 2, 64, 3.0, seed=8), "fp16x3") as m:
        spins = torch.zeros((B, 9), dtype=torch.uint8, device="cuda")
        assert f(m.handle, _p(spins), B, _p(e), None, None) == 6
    with rtt.RTT(inputs.workload("vhdd_6x6"), "fp32") as m:
        spins = torch.zeros((B, 36), dtype=torch.uint8, device="cuda")
        assert f(m.handle, _p(spins), B, _p(e), None, None) == 6
    with rtt.RTT(inputs.workload("tiny_fp64"), "fp64") as m:
        spins = torch.zeros((B, 9), dtype=torch.uint8, device="cuda")
        assert f(m.handle, None, B, _p(e), None, None) == 1
        assert f(m.handle, _p(spins), B, None, None, None) == 1
        assert f(m.handle, _p(spins), -1, _p(e), None, None) == 1
    torch.cuda.synchronize()
    assert torch.all(e == -2.0)
