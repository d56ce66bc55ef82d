"""Physical-space optimization (Sec. 3.2; Sec. 4, Table 1), composed from the
library's calls: every arithmetic step runs in librtt (kernels, or its host
solver for the small eigenproblem); this module only sequences them.

One iteration from the TT phi (psi = C phi):
  1. phi^alpha = O-bar_alpha phi for each operator (rtt_tt_apply: terms summed
     two by two, rounded to chi, scaled to unit norm);
  2. each phi^alpha becomes an RTT handle (b_L = b_R = e_0, the path of phi);
  3. dual Monte Carlo over the M states (rtt_dual_step): mixed local energies
     E^{ab} and ratios r^{ab} on samples of |psi^a|^2, averaged into H~, S~;
  4. H~ c = lambda S~ c (rtt_dual_solve), lowest eigenvalue;
  5. phi' = sum_alpha c_alpha phi^alpha rounded to chi (rtt_tt_sum_round).
"""
from __future__ import annotations

import numpy as np
import torch

from . import rtt


def lift_operators(n_spins: int, path, operators):
    """[(name, terms)] -> [(name, eta, ops)] through rtt_replica_lift.  An empty
    term list stands for the identity."""
    out = []
    L = len(path)
    for name, terms in operators:
        if not terms:
            out.append((name, np.ones(1), np.zeros((1, L), dtype=np.uint8)))
        else:
            eta, ops = rtt.replica_lift(n_spins, path, terms)
            out.append((name, eta, ops))
    return out


class PhysicalOptimizer:
    """Operators O_alpha (lifted), chi and the lattice of the states; precision
    is the sampler's (the operator states' handles), tt_precision the TT
    roundings' arithmetic (FP64 or FP32)."""

    def __init__(self, n_spins: int, path, bonds, J: float, h: float, chi: int, operators,
                 precision: str = "fp64", device: int = 0, tt_precision: str = "fp64"):
        self.n, self.path = int(n_spins), np.ascontiguousarray(path, dtype=np.int32)
        self.L = self.path.shape[0]
        self.bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
        self.J, self.h, self.chi = float(J), float(h), int(chi)
        self.precision, self.device = precision, device
        self.ops = lift_operators(self.n, self.path, operators)
        self.M = len(self.ops)
        self.plans = [rtt.TTPlan(self.L, self.chi, eta, ops, device, tt_precision)
                      for _, eta, ops in self.ops]
        self.comb = rtt.TTPlan(self.L, self.chi, np.ones(self.M),
                               np.zeros((self.M, self.L), dtype=np.uint8), device, tt_precision)

    def close(self):
        for p in self.plans:
            p.close()
        self.comb.close()

    def handle(self, cores: torch.Tensor, seed: int):
        """An RTT handle of psi = C phi for padded cores (device or host)."""
        from .inputs import RTTInstance
        e0 = np.zeros(self.chi)
        e0[0] = 1.0
        inst = RTTInstance(n_spins=self.n, path=self.path, tensors=cores.detach().cpu().numpy(),
                           b_left=e0, b_right=e0.copy(), bonds=self.bonds, J=self.J, h=self.h)
        return rtt.RTT(inst, self.precision, device=self.device, seed=seed)

    def operator_states(self, phi: torch.Tensor):
        """phi^alpha (device padded cores, unit norm) and log ||O-bar_alpha phi||."""
        phis, logn = [], torch.empty(self.M, dtype=torch.float64, device=phi.device)
        for a, plan in enumerate(self.plans):
            out = torch.empty_like(phi)
            plan.apply(phi, out, logn[a:a + 1])
            phis.append(out)
        return phis, logn

    def step(self, phi: torch.Tensor, spins0, chains: int, sweeps: int, burn: int, seed: int):
        """One iteration.  spins0: host uint8 [chains][N] starting configurations
        (the same for every state).  Returns a dict with the new cores 'phi',
        'lambda' (eigenvalues), 'c', 'Ht', 'St' and their standard errors."""
        phis, logn = self.operator_states(phi)
        hs = [self.handle(p, seed + 101 * a) for a, p in enumerate(phis)]
        M, B = self.M, chains
        sp = [torch.from_numpy(np.ascontiguousarray(spins0)).to(phi.device) for _ in range(M)]
        st = [h.log_amplitudes(x)[2] for h, x in zip(hs, sp)]
        for h, x, s in zip(hs, sp, st):
            h.mcmc_sweep(x, s, 0, burn)
        e = torch.empty((sweeps, M, M, B), dtype=torch.float64, device=phi.device)
        r = torch.empty_like(e)
        for t in range(sweeps):
            rtt.dual_step(hs, sp, st, burn + t, e[t], r[t])
        Ht, St, Hse, Sse = (np.zeros((M, M)) for _ in range(4))
        for a in range(M):
            for b in range(M):
                so = hs[a].observables(e[:, a, b, :].contiguous())
                sr = hs[a].observables(r[:, a, b, :].contiguous())
                Ht[a, b], Hse[a, b], St[a, b], Sse[a, b] = so["mean"], so["se"], sr["mean"], sr["se"]
        eig, c = rtt.dual_solve(Ht, St)
        new = torch.empty_like(phi)
        ln = torch.empty(1, dtype=torch.float64, device=phi.device)
        self.comb.sum_round(phis, c, new, ln)
        for h in hs:
            h.close()
        return {"phi": new, "lambda": eig, "c": c, "Ht": Ht, "St": St, "Ht_se": Hse, "St_se": Sse,
                "phis": phis, "log_norms": logn.cpu().numpy()}

    def energy(self, phi: torch.Tensor, chains: int, sweeps: int, burn: int, seed: int):
        """Sampled energy of psi = C phi: observables of E_loc (mean, se, v_score, ...)."""
        h = self.handle(phi, seed)
        from .inputs import initial_spins
        sp = torch.from_numpy(initial_spins(seed, chains, self.n)).to(phi.device)
        st = h.log_amplitudes(sp)[2]
        h.mcmc_sweep(sp, st, 0, burn)
        tr = torch.empty((sweeps, chains), dtype=torch.float64, device=phi.device)
        h.mcmc_sweep(sp, st, burn, sweeps, measure_every=1, trace=tr)
        obs = h.observables(tr)
        h.close()
        return obs
