"""Batched form: many FP32 instances of uneven N, R, chi in one persistent
launch.  Instance i must reproduce, bit for bit, a single-instance FP32 handle
of the same description (same row arithmetic in the same order, same Philox
stream per chain), whatever tile shape the autotuner picks and whether the
launch goes through the CUDA graph or not; sampled chains are checked against
the FP64 oracle."""
import json

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2604_22718_gb300 import inputs
from parity_util import eps_site, local_energy_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_22718_gb300 import build
    build.build()


def _small_batch():
    # the batched-workload generator on reduced lattices and chi
    return inputs.batched_instances(seed=7, n=9, chi_choices=(32, 64, 128), sizes=(4, 6),
                                    reps=(2, 3, 4))


def _single_reference(rtt, inst, seed, spins, n_steps, sweep0):
    B = spins.shape[0]
    with rtt.RTT(inst, "fp32", seed=seed) as m:
        sg = torch.from_numpy(spins.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        tr = torch.empty((n_steps, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, sweep0, n_steps, 1, tr, acc)
        torch.cuda.synchronize()
        return sg.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy(), acc.cpu().numpy()


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_single_instances_bit_for_bit(use_graph, tmp_path):
    from paper_2604_22718_gb300 import rtt
    insts = _small_batch()
    chains = [37 + 11 * i for i in range(len(insts))]       # ragged, not tile multiples
    seeds = [500 + i for i in range(len(insts))]
    n_steps = 3
    with rtt.RTTBatch(insts, chains, seeds=seeds) as b:
        if use_graph:
            b.tune(str(tmp_path / "tiles.json"), probe_chains=32)
        spins0 = np.concatenate([inputs.initial_spins(900 + i, c, inst.n_spins).ravel()
                                 for i, (inst, c) in enumerate(zip(insts, chains))])
        sp = torch.from_numpy(spins0.copy()).cuda()
        st = b.init(sp)
        e = torch.empty(b.total_chains, dtype=torch.float64, device="cuda")
        acc = torch.zeros(b.total_chains, dtype=torch.int64, device="cuda")
        traces = []
        for t in range(n_steps):
            b.step(sp, st, 4 + t, e, acc, use_graph=use_graph)
            traces.append(e.clone())
        torch.cuda.synchronize()
        tr = torch.stack(traces).cpu().numpy()
        sp, st, acc = sp.cpu().numpy(), st.cpu().numpy(), acc.cpu().numpy()
        shapes = [b.shape(i) for i in range(len(insts))]
    print("tile shapes", shapes)
    for i, inst in enumerate(insts):
        co, so = int(b.chain_off[i]), int(b.spin_off[i])
        B, N = chains[i], inst.n_spins
        s_ref, st_ref, tr_ref, acc_ref = _single_reference(
            rtt, inst, seeds[i], spins0[so:so + B * N].reshape(B, N), n_steps, 4)
        assert np.array_equal(sp[so:so + B * N].reshape(B, N), s_ref), i
        assert np.array_equal(st[co:co + B], st_ref), i
        assert np.array_equal(acc[co:co + B], acc_ref), i
        assert np.array_equal(tr[:, co:co + B], tr_ref), i
    if use_graph:
        cache = json.loads((tmp_path / "tiles.json").read_text())
        assert len(cache["tile_shapes"]) >= 1


def test_batch_sampled_chains_against_oracle():
    from paper_2604_22718_gb300 import rtt
    insts = _small_batch()[:3]
    chains = [64, 40, 50]
    with rtt.RTTBatch(insts, chains, seeds=[1, 2, 3]) as b:
        spins0 = np.concatenate([inputs.initial_spins(70 + i, c, inst.n_spins).ravel()
                                 for i, (inst, c) in enumerate(zip(insts, chains))])
        sp = torch.from_numpy(spins0.copy()).cuda()
        st = b.init(sp)
        e = torch.empty(b.total_chains, dtype=torch.float64, device="cuda")
        b.step(sp, st, 0, e)
        torch.cuda.synchronize()
        sp, e = sp.cpu().numpy(), e.cpu().numpy()
    for i, inst in enumerate(insts):
        o = orc.Oracle(inst)
        co, so, N = int(b.chain_off[i]), int(b.spin_off[i]), inst.n_spins
        pick = [0, chains[i] - 1]
        # the step measures the configuration it starts from
        s_in = spins0[so:so + chains[i] * N].reshape(chains[i], N)[pick]
        e_o = o.local_energies(s_in, threads=2)
        # FP32 rows: every ratio within |r| (chi + 1) u_32 (K(s) + K(s^(i)))
        _, r_o = o.local_energies(s_in, with_ratios=True, threads=2)
        bound = local_energy_bound(o, s_in, r_o, eps_site(inst.chi, "fp32"), inst.J, inst.h,
                                   inst.bonds.shape[0])
        assert np.all(np.abs(e[co + np.array(pick)] - e_o) <= bound), (i, e[co + np.array(pick)], e_o, bound)


def test_batch_chi256_and_12x12_r4_instances():
    """The batched workload's extremes in one launch: a chi = 256 instance (4x4,
    R = 2) and the largest lattice with the most replicas (12x12, R = 4, L =
    576, chi = 32).  Each reproduces a single FP32 handle bit for bit over two
    steps, and picked chains' measured energies lie within their FP32 bound of
    the FP64 oracle."""
    from paper_2604_22718_gb300 import rtt
    insts = [inputs.make_instance(4, 4, 2, 256, 3.1, seed=81), inputs.make_instance(12, 12, 4, 32, 2.7, seed=82)]
    chains = [40, 33]
    seeds = [11, 12]
    with rtt.RTTBatch(insts, chains, seeds=seeds) as b:
        spins0 = np.concatenate([inputs.initial_spins(83 + i, c, inst.n_spins).ravel()
                                 for i, (inst, c) in enumerate(zip(insts, chains))])
        sp = torch.from_numpy(spins0.copy()).cuda()
        st = b.init(sp)
        e = torch.empty(b.total_chains, dtype=torch.float64, device="cuda")
        acc = torch.zeros(b.total_chains, dtype=torch.int64, device="cuda")
        traces = []
        for t in range(2):
            b.step(sp, st, t, e, acc)
            traces.append(e.clone())
        torch.cuda.synchronize()
        tr = torch.stack(traces).cpu().numpy()
        sp, st, acc = sp.cpu().numpy(), st.cpu().numpy(), acc.cpu().numpy()
    for i, inst in enumerate(insts):
        co, so, B, N = int(b.chain_off[i]), int(b.spin_off[i]), chains[i], inst.n_spins
        s_in = spins0[so:so + B * N].reshape(B, N)
        s_ref, st_ref, tr_ref, acc_ref = _single_reference(rtt, inst, seeds[i], s_in, 2, 0)
        assert np.array_equal(sp[so:so + B * N].reshape(B, N), s_ref), i
        assert np.array_equal(st[co:co + B], st_ref), i
        assert np.array_equal(acc[co:co + B], acc_ref), i
        assert np.array_equal(tr[:, co:co + B], tr_ref), i
        o = orc.Oracle(inst)
        pick = [0, B - 1]
        e_o, r_o = o.local_energies(s_in[pick], with_ratios=True, threads=2)
        bound = local_energy_bound(o, s_in[pick], r_o, eps_site(inst.chi, "fp32"), inst.J, inst.h,
                                   inst.bonds.shape[0])
        print(inst.chi, inst.n_spins, "E_loc", tr[0, co + np.array(pick)], e_o, "bound", bound)
        assert np.all(np.abs(tr[0, co + np.array(pick)] - e_o) <= bound), i


def test_batch_rejects_unsupported_instances():
    from paper_2604_22718_gb300 import rtt
    tiny = inputs.make_instance(3, 3, 2, 8, 3.0, seed=1, mixing=False)
    with pytest.raises(rtt.RTTError):
        rtt.RTTBatch([tiny], [4])                                   # chi < 17 on the CUDA cores
    small = inputs.make_instance(3, 3, 2, 32, 3.0, seed=2)
    with pytest.raises(rtt.RTTError):
        rtt.RTTBatch([small], [4], precisions=["fp64"])             # FP64 is not batched
    with pytest.raises(rtt.RTTError):
        rtt.RTTBatch([small], [4], precisions=["fp16x3"])           # tensor cores need chi 64 or 128


def _single_reference_prec(rtt, inst, prec, seed, spins, n_steps, sweep0):
    B = spins.shape[0]
    with rtt.RTT(inst, prec, seed=seed) as m:
        sg = torch.from_numpy(spins.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        tr = torch.empty((n_steps, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        for t in range(n_steps):
            m.mcmc_sweep(sg, st, sweep0 + t, 1, 1, tr[t:t + 1], acc)
        torch.cuda.synchronize()
        return sg.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy(), acc.cpu().numpy()


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_tensor_core_instances(use_graph):
    """FP16X3 instances (chi 64 and 128) beside FP32 ones: every instance
    reproduces a single handle of its own precision bit for bit over three
    steps (ragged chain counts), and the tensor-core instances' measured
    energies lie within their split bound of the FP64 oracle."""
    from paper_2604_22718_gb300 import rtt
    insts = [inputs.make_instance(4, 4, 2, 32, 3.0, seed=91), inputs.make_instance(4, 4, 3, 64, 2.9, seed=92),
             inputs.make_instance(4, 4, 2, 128, 3.1, seed=93), inputs.make_instance(3, 4, 2, 128, 3.0, seed=94)]
    precs = ["fp32", "fp16x3", "fp16x3", "fp32"]
    chains = [45, 150, 70, 33]
    seeds = [21, 22, 23, 24]
    n_steps = 3
    with rtt.RTTBatch(insts, chains, seeds=seeds, precisions=precs) as b:
        spins0 = np.concatenate([inputs.initial_spins(95 + i, c, inst.n_spins).ravel()
                                 for i, (inst, c) in enumerate(zip(insts, chains))])
        sp = torch.from_numpy(spins0.copy()).cuda()
        st = b.init(sp)
        e = torch.empty(b.total_chains, dtype=torch.float64, device="cuda")
        acc = torch.zeros(b.total_chains, dtype=torch.int64, device="cuda")
        traces = []
        for t in range(n_steps):
            b.step(sp, st, 7 + t, e, acc, use_graph=use_graph)
            traces.append(e.clone())
        torch.cuda.synchronize()
        tr = torch.stack(traces).cpu().numpy()
        sp, st, acc = sp.cpu().numpy(), st.cpu().numpy(), acc.cpu().numpy()
    for i, inst in enumerate(insts):
        co, so, B, N = int(b.chain_off[i]), int(b.spin_off[i]), chains[i], inst.n_spins
        s_in = spins0[so:so + B * N].reshape(B, N)
        s_ref, st_ref, tr_ref, acc_ref = _single_reference_prec(rtt, inst, precs[i], seeds[i], s_in, n_steps, 7)
        assert np.array_equal(sp[so:so + B * N].reshape(B, N), s_ref), i
        assert np.array_equal(st[co:co + B], st_ref), i
        assert np.array_equal(acc[co:co + B], acc_ref), i
        assert np.array_equal(tr[:, co:co + B], tr_ref), i
        if precs[i] == "fp16x3":
            o = orc.Oracle(inst)
            pick = [0, B - 1]
            e_o, r_o = o.local_energies(s_in[pick], with_ratios=True, threads=2)
            bound = local_energy_bound(o, s_in[pick], r_o, eps_site(inst.chi, "fp16x3"), inst.J, inst.h,
                                       inst.bonds.shape[0])
            assert np.all(np.abs(tr[0, co + np.array(pick)] - e_o) <= bound), i
