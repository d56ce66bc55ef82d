"""Physical-space optimization (Sec. 3.2; Sec. 4, Table 1), composed from the
library's calls: every arithmetic step runs in librtt (kernels, or its host
solver for the small eigenproblem); this module only sequences them.

One iteration from the TT phi of rank chi (psi = C phi):
  1. phi^alpha = O-bar_alpha phi for each operator (rtt_tt_apply: terms summed
     two by two, kept at the state rank chi_s, scaled to unit norm);
  2. each phi^alpha becomes an RTT handle (b_L = b_R = e_0, the path of phi);
  3. dual Monte Carlo over the M states (rtt_dual_step): mixed local energies
     E^{ab} and ratios r^{ab} on samples of |psi^a|^2, averaged into H~, S~;
  4. H~ c = lambda S~ c (rtt_dual_solve), lowest eigenvalue;
  5. phi' = sum_alpha c_alpha phi^alpha compressed back to chi
     (rtt_tt_sum_round).
With gram_schmidt set (Sec. 3.3, Eq. Gram-Schmid), a short pilot pass gives S~
on the states psi^alpha (against psi^1 only: chains of psi^1 alone and their
ratios to the others; otherwise a pilot of step 3); step 3 then runs on
psi'^m = psi^m - sum_{a<m} S~_{am} psi^a (or a = 1 only), each an exact
direct-sum RTT (rtt_create_sum), so that the overlap matrix the eigenproblem
sees is close to diagonal; step 4 gives c' in that basis and step 5 combines
the phi^alpha with c = T^T c' (psi' = T psi).
Sec. 3.2 compresses only the final combination; the operator states keep the
rank chi_s = 2 chi (the rank of a sum of two rank-chi TTs) by default, so the
eigenproblem sees O_alpha psi rather than its rank-chi truncation.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import rtt


class _PhaseClock:
    """Host wall time of each phase of an iteration, the device synchronized
    at every mark (the phases are sequential anyway: each one's results go
    through the host)."""

    def __init__(self):
        torch.cuda.synchronize()
        self.t = time.perf_counter()
        self.phases = {}

    def mark(self, name):
        torch.cuda.synchronize()
        now = time.perf_counter()
        self.phases[name] = now - self.t
        self.t = now


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
    roundings' arithmetic (FP64 or FP32); chi_states the operator states' rank
    (0: min(2 chi, 16)), the tree sums inside each O-bar_alpha phi rounded to
    min(2 chi_states, 16)."""

    def __init__(self, n_spins: int, path, bonds, J: float, h: float, chi: int, operators,
                 precision: str = "fp64", device: int = 0, tt_precision: str = "fp64",
                 chi_states: int = 0):
        self.n, self.path = int(n_spins), np.ascontiguousarray(path, dtype=np.int32)
        self.L = self.path.shape[0]
        self.bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
        self.J, self.h, self.chi = float(J), float(h), int(chi)
        self.precision, self.device = precision, device
        self.ops = lift_operators(self.n, self.path, operators)
        self.M = len(self.ops)
        self.chi_s = int(chi_states) or min(2 * self.chi, 16)
        if not self.chi <= self.chi_s <= 16:
            raise ValueError("chi_states must be in [chi, 16]")
        self.plans = [rtt.TTPlan(self.L, self.chi_s, eta, ops, device, tt_precision,
                                 chi_tree=min(2 * self.chi_s, 16)) for _, eta, ops in self.ops]
        self._streams = []
        self.comb = rtt.TTPlan(self.L, self.chi, np.ones(self.M),
                               np.zeros((self.M, self.L), dtype=np.uint8), device, tt_precision,
                               chi_tree=self.chi_s)

    def close(self):
        for p in self.plans:
            p.close()
        self.comb.close()

    def instance(self, cores: torch.Tensor):
        """The RTT description of psi = C phi for padded cores [L][2][c][c]
        (device or host): b_L = b_R = e_0 on the path of phi."""
        from .inputs import RTTInstance
        e0 = np.zeros(int(cores.shape[2]))
        e0[0] = 1.0
        return RTTInstance(n_spins=self.n, path=self.path, tensors=cores.detach().cpu().numpy(),
                           b_left=e0, b_right=e0.copy(), bonds=self.bonds, J=self.J, h=self.h)

    def handle(self, cores: torch.Tensor, seed: int):
        """An RTT handle of psi = C phi for padded cores [L][2][c][c] (device or host)."""
        return rtt.RTT(self.instance(cores), self.precision, device=self.device, seed=seed)

    def operator_states(self, phi: torch.Tensor):
        """phi^alpha (device padded cores of rank chi_s, unit norm) and
        log ||O-bar_alpha phi||."""
        phis, logn = [], torch.empty(self.M, dtype=torch.float64, device=phi.device)
        shape = (self.L, 2, self.chi_s, self.chi_s)
        # the operators are independent (own plans, node buffers and scratch):
        # each tree runs on its own stream, a few warps per level each
        cur = torch.cuda.current_stream(phi.device)
        if len(self._streams) < self.M:
            self._streams = [torch.cuda.Stream(phi.device) for _ in range(self.M)]
        for a, plan in enumerate(self.plans):
            out = torch.empty(shape, dtype=torch.float64, device=phi.device)
            st = self._streams[a]
            st.wait_stream(cur)
            plan.apply(phi, out, logn[a:a + 1], stream=st)
            phis.append(out)
        for a in range(self.M):
            cur.wait_stream(self._streams[a])
        return phis, logn

    def combine(self, phis, coef):
        """phi' = sum_alpha coef[alpha] phi^alpha compressed to chi and scaled to
        unit norm (Eq. lin_comb; rtt_tt_sum_round), phis of rank chi_s."""
        new = torch.empty((self.L, 2, self.chi, self.chi), dtype=torch.float64,
                          device=phis[0].device)
        self.comb.sum_round(phis, coef, new)
        return new

    def _dual(self, hs, spins0, sweeps: int, burn: int, device, sweep0: int = 0):
        """Dual Monte Carlo over the handles: burn-in sweeps, then one dual step
        per sweep (the sweeps numbered from sweep0 for the random streams);
        H~, S~ and their standard errors."""
        M = len(hs)
        B = int(np.asarray(spins0).shape[0])
        sp = [torch.from_numpy(np.ascontiguousarray(spins0)).to(device) for _ in range(M)]
        st = [h.log_amplitudes(x)[2] for h, x in zip(hs, sp)]
        for h, x, s in zip(hs, sp, st):
            h.mcmc_sweep(x, s, sweep0, burn)
        e = torch.empty((sweeps, M, M, B), dtype=torch.float64, device=device)
        r = torch.empty_like(e)
        for t in range(sweeps):
            rtt.dual_step(hs, sp, st, sweep0 + burn + t, e[t], r[t])
        Ht, St, Hse, Sse = (np.zeros((M, M)) for _ in range(4))
        for a in range(M):
            for b in range(M):
                so = hs[a].observables(e[:, a, b, :].contiguous())
                sr = hs[a].observables(r[:, a, b, :].contiguous())
                Ht[a, b], Hse[a, b], St[a, b], Sse[a, b] = so["mean"], so["se"], sr["mean"], sr["se"]
        return Ht, St, Hse, Sse

    def _pilot_first(self, hs, spins0, sweeps: int, burn: int, device):
        """S~_{0m} = <psi^m / psi^1>_{P^1} (the only overlaps the Gram-Schmidt
        against psi^1 needs) from chains of psi^1 alone: burn-in, then per sweep
        the ratios psi^m / psi^1 at its configurations.  Row 0 of S~ and its
        standard errors; the other rows are NaN."""
        M = len(hs)
        h0 = hs[0]
        sp = torch.from_numpy(np.ascontiguousarray(spins0)).to(device)
        st = h0.log_amplitudes(sp)[2]
        h0.mcmc_sweep(sp, st, 0, burn)
        r = torch.empty((M, sweeps, sp.shape[0]), dtype=torch.float64, device=device)
        for t in range(sweeps):
            h0.mcmc_sweep(sp, st, burn + t, 1)
            for m in range(1, M):
                r[m, t] = h0.mixed_local_energy(hs[m], sp)[1]
        St, Sse = np.full((M, M), np.nan), np.full((M, M), np.nan)
        St[0, 0], Sse[0, 0] = 1.0, 0.0
        for m in range(1, M):
            o = h0.observables(r[m])
            St[0, m], Sse[0, m] = o["mean"], o["se"]
        return St, Sse

    @staticmethod
    def gram_schmidt_matrix(St, first_only: bool):
        """T of psi' = T psi for Eq. Gram-Schmid (rtt_dual_gram_schmidt): row m
        holds 1 at m and -<psi^m / psi^a>_{P^a} = -S~_{am} at every a < m
        (a = 0 only when first_only)."""
        return rtt.dual_gram_schmidt(St, first_only)

    def step(self, phi: torch.Tensor, spins0, chains: int, sweeps: int, burn: int, seed: int,
             gram_schmidt: str = "", pilot_sweeps: int = 0):
        """One iteration.  spins0: host uint8 [chains][N] starting configurations
        (the same for every state).  gram_schmidt: "" (none), "first" or "all"
        (Eq. Gram-Schmid against psi^1 only, or against every earlier state),
        its S~ from a pilot pass of pilot_sweeps (0: max(sweeps // 5, 10))
        sweeps.  Returns a dict with the new cores 'phi', 'lambda'
        (eigenvalues), 'c' (on the phi^alpha), 'Ht', 'St' and their standard
        errors (in the basis the dual Monte Carlo ran on), 'T' (that basis:
        psi' = T psi; the identity without Gram-Schmidt) and, with
        Gram-Schmidt, 'pilot_St' and 'pilot_St_se' (only row 0 for "first")."""
        if gram_schmidt not in ("", "first", "all"):
            raise ValueError("gram_schmidt must be '', 'first' or 'all'")
        clock = _PhaseClock()
        phis, logn = self.operator_states(phi)
        clock.mark("operator_states")
        hs = [self.handle(p, seed + 101 * a) for a, p in enumerate(phis)]
        clock.mark("handles")
        M = self.M
        T = np.eye(M)
        pilot = None
        if gram_schmidt and M > 1:
            ps = int(pilot_sweeps) or max(sweeps // 5, 10)
            if gram_schmidt == "first":
                pilot_St, pilot_se = self._pilot_first(hs, spins0, ps, burn, phi.device)
            else:
                _, pilot_St, _, pilot_se = self._dual(hs, spins0, ps, burn, phi.device)
            pilot = (pilot_St, pilot_se)
            clock.mark("pilot")
            T = self.gram_schmidt_matrix(pilot_St, gram_schmidt == "first")
            insts = [self.instance(p) for p in phis]
            for m in range(1, M):
                used = [a for a in range(M) if T[m, a] != 0.0]
                gs = rtt.RTT.from_sum([insts[a] for a in used], T[m, used], self.precision,
                                      device=self.device, seed=seed + 101 * m + 7)
                hs[m].close()
                hs[m] = gs
            clock.mark("gram_schmidt_handles")
        Ht, St, Hse, Sse = self._dual(hs, spins0, sweeps, burn, phi.device,
                                      0 if pilot is None else burn + ps)
        clock.mark("dual_monte_carlo")
        eig, cp = rtt.dual_solve(Ht, St)
        c = rtt.dual_back_transform(T, cp) if pilot is not None else cp
        new = self.combine(phis, c)
        clock.mark("solve_and_combine")
        for h in hs:
            h.close()
        out = {"phi": new, "lambda": eig, "c": c, "Ht": Ht, "St": St, "Ht_se": Hse, "St_se": Sse,
               "T": T, "phis": phis, "log_norms": logn.cpu().numpy(), "timing": clock.phases}
        if pilot is not None:
            out["pilot_St"], out["pilot_St_se"] = pilot
        return out

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
