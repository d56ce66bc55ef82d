/*
 * rtt.h -- C ABI of the GB300 replica-tensor-train (RTT) Monte Carlo library.
 *
 * An RTT (arxiv 2604.22718, Sec. 2.2.1, Eq. RTT) is a tensor train of length
 * L whose site k carries two chi x chi matrices A_k[0], A_k[1] and is tied to
 * physical spin path[k]:
 *
 *     psi(s) = b_L^T A_0[s_path(0)] A_1[s_path(1)] ... A_{L-1}[s_path(L-1)] b_R
 *
 * (the trace of Eq. RTT with the first and last bond of dimension one, Sec.
 * 2.1, written with boundary vectors b_L, b_R).  The library samples
 * P(s) = |psi(s)|^2 / Z with single-spin Metropolis (Sec. 3.3) over many
 * independent chains and evaluates the transverse-field Ising local energy
 *
 *     E_loc(s) = J sum_<ij> z_i z_j - h sum_i psi(s^(i)) / psi(s)
 *
 * (Sec. 3.3, mixed local energy with psi^1 = psi^2; Hamiltonian Sec. 4, Eq.
 * ising-model), z_i = 1 - 2 s_i, s^(i) = s with spin i flipped.
 *
 * Conventions shared by all calls
 *   - Spins are uint8 in {0,1}, row-major [B][N] (chain-major).
 *   - Pointers documented "device" must be device memory of the handle's GPU;
 *     "host" pointers are read before the call returns.
 *   - Every call is asynchronous and ordered on `stream` (a cudaStream_t;
 *     NULL = the legacy default stream) unless documented otherwise.
 *   - Amplitudes are kept as psi = mant * 2^exp2 with |mant| in [1,2); the
 *     exponent is an exact integer sum of per-site power-of-two rescalings, so
 *     no train length over- or underflows.
 *   - Paths: L = R N sites with path[0..N-1] a permutation of the N spins;
 *     Metropolis proposal j of a sweep flips spin path[j] (systematic scan).
 *     Periodic paths, path[k] = path[k mod N] (an ordering repeated R times),
 *     run everywhere.  General paths (the replicas visit the spins in
 *     different orders, e.g. sigma^V + sigma^H + sigma^D + sigma^D' -- the
 *     path sums of Sec. 2.2.1) run on FP64/FP32 handles, and on BF16X3/FP16X3
 *     handles for amplitudes and local energies and, with R >= 2, for sweeps
 *     (at chi = 128 when the batch's CTA pairs, two SMs per 128 chains, fit on
 *     the GPU at once; RTT_ERR_UNSUPPORTED otherwise); the batched form and
 *     rtt_local_energy_noalloc need periodic
 *     paths.  Each flip row of a general path spans its spin's first to last
 *     site, and a sweep rebuilds the part after the last site per proposal.
 *   - Errors: argument errors are detected before anything is launched and
 *     leave all outputs untouched; CUDA errors (including asynchronous ones of
 *     earlier launches on the device) return RTT_ERR_CUDA.  rtt_last_error()
 *     gives a message for the calling thread.  No call aborts the process.
 */
#ifndef RTT_H
#define RTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtt_s *rtt_handle;

typedef enum {
    RTT_OK = 0,
    RTT_ERR_INVALID_ARG = 1,
    RTT_ERR_CUDA = 2,
    RTT_ERR_OOM = 3,
    RTT_ERR_NUMERIC = 4,
    RTT_ERR_TIMEOUT = 5,
    RTT_ERR_UNSUPPORTED = 6
} rtt_status;

/* Arithmetic of the site contractions (exponents are always exact integers,
 * energies and statistics are always reduced in FP64). */
typedef enum {
    RTT_FP64 = 0,   /* FP64 fma chains in the oracle's canonical order         */
    RTT_FP32 = 1,   /* FP32 fma chains                                         */
    RTT_BF16X3 = 2, /* tensor cores: bf16 hi/lo split operands, 3 products
                       (hi*hi + hi*lo + lo*hi), FP32 accumulation             */
    RTT_FP16X3 = 3  /* as RTT_BF16X3 with fp16 hi/lo operands (11-bit
                       significands; site tensors prescaled by exact powers
                       of two into fp16's normal range)                       */
} rtt_precision;

typedef struct {
    int32_t n_spins;          /* N >= 1                                          */
    int32_t length;           /* L = number of train sites, a multiple of N      */
    int32_t chi;              /* bond dimension, 1..256                          */
    int32_t n_bonds;          /* number of ZZ bonds (may be 0)                   */
    const int32_t *path;      /* host [L]; path[k] in [0,N)                      */
    const double *tensors;    /* host [L][2][chi][chi]; A_k[s][a][b], finite     */
    const double *b_left;     /* host [chi]                                      */
    const double *b_right;    /* host [chi]                                      */
    const int32_t *bonds;     /* host [n_bonds][2] spin pairs (i != j)           */
    double J;                 /* ZZ coupling                                     */
    double h;                 /* transverse field                                */
    int32_t precision;        /* rtt_precision                                   */
    int32_t device;           /* CUDA device ordinal, or -1 for the current one  */
    uint64_t seed;            /* key of the Metropolis random stream             */
} rtt_desc;

/* psi = mant * 2^exp2, |mant| in [1,2) or mant == 0. */
typedef struct {
    double mant;
    int64_t exp2;
} rtt_chain_state;

/* Summary statistics of a local-energy trace (rtt_observables). */
typedef struct {
    double mean;         /* grand mean of E_loc                                     */
    double var;          /* (1/n) sum (E_loc - mean)^2                              */
    double se;           /* sqrt(var * 2 tau_int / n)                               */
    double se_bin;       /* binned SE, bins of ceil(20 tau_int) sweeps per chain    */
    double se_chain;     /* std of chain means / sqrt(B)                            */
    double tau_int;      /* 1/2 + sum_{t<=W} rho(t), Sokal window W >= 5 tau(W)     */
    double ess;          /* n / (2 tau_int)                                         */
    double v_score;      /* N var / mean^2 (Sec. 4.3, Table 1 and Fig. 6)           */
    double accept_rate;  /* accepted / proposed, NaN if no counts given             */
    int64_t n;           /* T * B                                                   */
    int32_t window;      /* W                                                       */
    int32_t pad;
} rtt_stats;

/* Create a handle: validates the description (path as above, finite tensors,
 * bond indices in range), copies every host array to the device in the
 * requested precision and returns the handle in *out.  The handle owns its
 * device copies and its scratch; the caller keeps ownership of `desc` and its
 * arrays.  Unsupported combinations (first N sites not a permutation,
 * chi > 256, BF16X3 or FP16X3 with chi not in {64,128}) return
 * RTT_ERR_UNSUPPORTED. */
rtt_status rtt_create(const rtt_desc *desc, rtt_handle *out);

/* Release every device allocation of the handle (synchronises its device). */
rtt_status rtt_destroy(rtt_handle h);

/* Pre-allocate the scratch used for batches of up to B chains so that later
 * calls with B' <= B allocate nothing.  Scratch grows on demand otherwise. */
rtt_status rtt_reserve(rtt_handle h, int64_t B);

/* log|psi(s)| and sign for B configurations (Eq. RTT, evaluated left to
 * right).  spins: device [B][N]; log_abs: device [B] (-inf where psi = 0);
 * sign: device int8 [B] (+1, -1, 0); state: device [B] or NULL, receives
 * (mant, exp2) -- the chain state rtt_mcmc_sweep expects. */
rtt_status rtt_log_amplitudes(rtt_handle h, const uint8_t *spins, int64_t B,
                              double *log_abs, int8_t *sign, rtt_chain_state *state,
                              void *stream);

/* Local energy E_loc(s) for B configurations (Sec. 3.3 with Sec. 4 Eq.
 * ising-model).  psi(s^(i)) is evaluated by the factorisation
 * l_{a-1} A_a .. A_b r_{b+1} over the replica span [a,b] of spin i using
 * cached left (first N sites) and right (last N sites) environments; psi(s)
 * by a full left-to-right pass.  spins: device [B][N]; e_loc: device [B]
 * (NaN where psi(s) = 0); ratios: device [B][N] or NULL, receives
 * psi(s^(i))/psi(s) indexed by spin i. */
rtt_status rtt_local_energy(rtt_handle h, const uint8_t *spins, int64_t B, double *e_loc,
                            double *ratios, void *stream);

/* Run n_sweeps systematic single-spin Metropolis sweeps on B chains (Sec. 3.3:
 * sampling of P(s) = |psi(s)|^2/Z).  Proposal j of sweep t flips spin path[j]
 * and is accepted iff u < (psi(s')/psi(s))^2 with
 * u = (Philox4x64-10(counter = (chain0+c, t, j, 0), key = (seed, 0x4D434D43))[0] >> 11) * 2^-53,
 * t = sweep0 + sweep index, so a run split into several calls, or chains split
 * across calls by chain0, reproduces the unsplit run bit for bit in FP64.
 *   spins     device [B][N]   in/out
 *   state     device [B]      in/out, psi of the current spins (from
 *                             rtt_log_amplitudes), updated on acceptance
 *   e_loc_trace device [n_sweeps/measure_every][B] or NULL (measure_every >= 1):
 *             row g holds E_loc of the configuration entering sweep
 *             g*measure_every of this call -- each measured iteration
 *             evaluates the configuration it starts from, then runs its
 *             measure_every sweeps; trailing sweeps are not measured.  The
 *             library evaluates it on a second, internal stream from a copy
 *             of the spins, concurrently with the sweeps; all of the call's
 *             work is ordered before later work on `stream`.
 *   n_accept  device int64 [B] or NULL: accepted proposals are added
 * Chains whose psi is 0 or not finite accept any proposal with a finite,
 * nonzero amplitude. */
rtt_status rtt_mcmc_sweep(rtt_handle h, uint8_t *spins, rtt_chain_state *state, int64_t B,
                          int64_t chain0, int64_t sweep0, int32_t n_sweeps, int32_t measure_every,
                          double *e_loc_trace, int64_t *n_accept, void *stream);

/* Statistics of a local-energy trace (V-score of Sec. 4.3; tau_int by Sokal's
 * automatic window with c = 5).  e_loc_trace: device [T][B]; n_accept: device
 * [B] or NULL; proposals_per_chain: divisor of the acceptance rate; out: host.
 * SYNCHRONOUS: returns after the device work on `stream` has finished. */
rtt_status rtt_observables(rtt_handle h, const double *e_loc_trace, int32_t T, int64_t B,
                           const int64_t *n_accept, int64_t proposals_per_chain, rtt_stats *out,
                           void *stream);

/* ---------------------------------------------------------------------------
 * Dual Monte Carlo (Sec. 3.3): matrix elements between M RTT states psi^1..psi^M
 * of one lattice, each sampled from its own P^a = |psi^a|^2 / Z_a.
 *
 * Mixed local energy and overlap ratio of configurations s (typically drawn
 * from P^a by rtt_mcmc_sweep on handle a):
 *   E^{ab}(s) = sum_sbar H_{s,sbar} psi^b(sbar) / psi^a(s)
 *             = [J sum_<ij> z_i z_j psi^b(s) - h sum_i psi^b(s^(i))] / psi^a(s)
 *   r^{ab}(s) = psi^b(s) / psi^a(s)
 * so that H~_ab = <E^{ab}>_{P^a} and S~_ab = <r^{ab}>_{P^a} (the un-symmetrised
 * matrices of Eq. gen_eig2; rtt_observables gives their means and errors).
 * Each amplitude ratio is ldexp(mant_b / mant_a, exp_b - exp_a); the field term
 * adds the N flip ratios in increasing spin index; E = (J zz) r - h sum, all in
 * FP64 (bit-identical to the FP64 oracle for FP64 handles).  Handles a and b
 * (a may equal b, giving E_loc and r = 1) must be on one device and share N, the
 * bond list, J and h; their tensors, R, chi and precision may differ.
 *   spins   device [B][N]
 *   e_mixed device [B]
 *   ratio   device [B] or NULL
 * Configurations with psi^a(s) zero or not finite give NaN.  Asynchronous on
 * `stream`; uses both handles' scratch. */
rtt_status rtt_mixed_local_energy(rtt_handle a, rtt_handle b, const uint8_t *spins, int64_t B,
                                  double *e_mixed, double *ratio, void *stream);

/* One dual Monte Carlo iteration for M states (Sec. 3.3): for every state a, the
 * mixed local energies E^{ab} and ratios r^{ab} (all b) of the configurations
 * a's chains enter the iteration with (as rtt_mixed_local_energy), then one
 * systematic sweep of a's chains on P^a (as rtt_mcmc_sweep with chain0 and
 * sweep0 = sweep).  The measurements run from copies of the spins on the
 * handles' second streams, in M waves: wave w evaluates the pairs (a, (a+w)
 * mod M), so that no two concurrent pairs share a handle's energy scratch;
 * with FP64/FP32 handles each state's sweep runs on its own handle's third
 * stream, so the M sweeps and the measurements proceed side by side
 * (tensor-core sweeps, which fill 64 SMs per 4096 chains, run one after
 * another on `stream`); all work is ordered after earlier and before later
 * work on `stream`.  The M handles must be distinct; calls on one set of
 * handles must not overlap (they share the handles' streams and scratch).
 *   handles   host [M] (M >= 1), one lattice as for rtt_mixed_local_energy
 *   spins     host [M] of device [B][N]; state host [M] of device [B]
 *   e_mixed   device [M][M][B] (a-major, then b) or NULL; ratio likewise
 *   n_accept  host [M] of device [B] or NULL (as may be every entry) */
rtt_status rtt_dual_step(const rtt_handle *handles, int32_t M, uint8_t *const *spins,
                         rtt_chain_state *const *state, int64_t B, int64_t chain0, int64_t sweep,
                         double *e_mixed, double *ratio, int64_t *const *n_accept, void *stream);

/* One RTT for a linear combination psi(s) = sum_m coef[m] psi^m(s) of M RTTs on
 * the same path (Sec. 3.2: psi' is turned back into an RTT by summing tensor
 * trains; the stochastic Gram-Schmidt states of Sec. 3.3, Eq. Gram-Schmid, are
 * such combinations).  A sum of TTs is a TT: site tensors block-diagonal,
 * A_k[s] = diag(A^1_k[s], ..., A^M_k[s]); b_R = (b^1_R, ..., b^M_R);
 * b_L = (coef[0] b^1_L, ..., coef[M-1] b^M_L).  All descriptions must share
 * n_spins, length, path, bonds, J and h; chi = sum of the chi_m (<= 256, and
 * 64 or 128 for the tensor-core precisions); precision, device and seed are
 * those of descs[0].  descs: host [M]; coef: host [M]; *out as rtt_create. */
rtt_status rtt_create_sum(const rtt_desc *descs, int32_t M, const double *coef, rtt_handle *out);

/* Generalized eigenproblem H~ c = lambda S~ c of Eq. gen_eig2 (Sec. 3.3), whose
 * lowest eigenvalue is the energy of the optimal combination sum_a c_a psi^a.
 * Solved as the eigenvalues of S~^-1 H~ (LU with partial pivoting, Householder
 * Hessenberg reduction, shifted complex QR), host FP64.
 *   M       1..8
 *   Ht, St  host [M][M] row-major, (H~_ab, S~_ab)
 *   eig_re, eig_im  host [M]: eigenvalues by increasing real part (ties by
 *           imaginary part)
 *   c0      host [M] or NULL: for a real lowest eigenvalue (|Im| <= 1e-9 max|lambda|)
 *           its eigenvector (inverse iteration on S~^-1 H~), scaled to
 *           |c^T S~ c| = 1 with its largest-magnitude entry positive; NaN otherwise
 * RTT_ERR_NUMERIC if S~ is singular or the QR iteration does not converge.
 * Host computation only; no device work, callable without a GPU. */
rtt_status rtt_dual_solve(int32_t M, const double *Ht, const double *St, double *eig_re,
                          double *eig_im, double *c0);

/* The stochastic Gram-Schmidt basis of Sec. 3.3 (Eq. Gram-Schmid):
 * psi'^m = psi^m - sum_a <psi^m / psi^a>_{P^a} psi^a over a < m (a = 0 only
 * when first_only != 0), <psi^m / psi^a>_{P^a} = S~_am.  Writes T (host
 * [M][M] row-major) with psi' = T psi: T[m][m] = 1, T[m][a] = -S~[a][m].
 * St: host [M][M]; 1 <= M <= 8; RTT_ERR_NUMERIC on a non-finite entry used.
 * Host computation only. */
rtt_status rtt_dual_gram_schmidt(int32_t M, const double *St, int32_t first_only, double *T);

/* Coefficients on the original states from those on psi' = T psi:
 * c = T^T c' (sum over m in increasing order).  T: host [M][M] row-major;
 * c_prime, c: host [M], c must not alias c_prime; 1 <= M <= 8.  Host
 * computation only. */
rtt_status rtt_dual_back_transform(int32_t M, const double *T, const double *c_prime, double *c);

/* The Metropolis uniforms themselves, for checking the device generator:
 * counters: device uint64 [n][3] = (chain, sweep, proposal); out: device [n]. */
rtt_status rtt_mcmc_uniforms(uint64_t seed, int64_t n, const uint64_t *counters, double *out,
                             void *stream);

/* Per-kernel device time.  While profiling is enabled, the library brackets
 * every kernel it launches for this handle with a pair of CUDA events on the
 * launching stream.  rtt_profile_read synchronises the handle's device, writes
 * up to `capacity` entries (one per kernel kind that ran: static name, number
 * of launches, summed milliseconds), stores the number of kinds in *count and
 * resets the counters.  Enabling or disabling also resets them. */
typedef struct {
    const char *name;
    int64_t launches;
    double ms;
} rtt_kernel_time;
rtt_status rtt_profile(rtt_handle h, int32_t enable);
rtt_status rtt_profile_read(rtt_handle h, rtt_kernel_time *out, int32_t capacity, int32_t *count);

/* ---------------------------------------------------------------------------
 * Batched form: many independent RTT instances of uneven N, R and chi sampled
 * together.  Each instance is an rtt_desc (periodic path, all on one device)
 * and gets its own chains.  FP32 instances (17 <= chi <= 256) run on the CUDA
 * cores in ONE persistent kernel launch per iteration (optionally through a
 * CUDA graph); FP16X3 / BF16X3 instances (chi in {64, 128}) run on the tensor
 * cores, each as one rtt_mcmc_sweep of its own handle on the same stream after
 * that launch.  One call of rtt_batch_step performs one Monte Carlo iteration
 * of every chain of every instance -- the local energy of the configuration
 * it starts from (Sec. 3.3 / Sec. 4 Eq. ising-model), then one systematic
 * sweep (Sec. 3.3).  Results of instance i equal, bit for bit, those of an
 * rtt_handle of the same description running rtt_mcmc_sweep with chain0 = 0,
 * sweep0 = sweep, measure_every = 1.
 *
 * Device buffers are packed instance after instance: spins [sum_i B_i N_i]
 * (instance i at spin offset so_i, chain c at so_i + c N_i), chain state and
 * e_loc [sum_i B_i] (instance i at chain offset co_i); rtt_batch_layout returns
 * the offsets.  The batch owns its per-instance handles and scratch.
 * --------------------------------------------------------------------------- */
typedef struct rtt_batch_s *rtt_batch;
rtt_status rtt_batch_create(const rtt_desc *descs, int32_t n_instances, const int64_t *chains,
                            rtt_batch *out);
rtt_status rtt_batch_destroy(rtt_batch b);
/* totals and per-instance offsets (host arrays of n_instances, or NULL) */
rtt_status rtt_batch_layout(rtt_batch b, int64_t *total_chains, int64_t *total_spins,
                            int64_t *chain_off, int64_t *spin_off);
/* chain states (psi of the current spins) of every instance, Eq. RTT */
rtt_status rtt_batch_init(rtt_batch b, const uint8_t *spins, rtt_chain_state *state, void *stream);
/* one iteration (sweep index `sweep`) of every chain; e_loc [sum B_i] receives
 * E_loc of the configuration the iteration starts from (measured before its
 * sweep, as rtt_mcmc_sweep measures); n_accept [sum B_i] (or NULL)
 * accumulates acceptances.
 * use_graph != 0 launches the persistent kernel through a CUDA graph built on
 * first use (its kernel node is updated per call). */
rtt_status rtt_batch_step(rtt_batch b, uint8_t *spins, rtt_chain_state *state, int64_t sweep,
                          double *e_loc, int64_t *n_accept, int32_t use_graph, void *stream);
/* Autotuner: for every (chi, L) bucket (L <= 64, <= 256, > 256) time each tile
 * shape -- 32 or 16 lanes per row, 1 or 2 blocks of rows per work item -- on
 * up to probe_chains chains per instance of the bucket and keep the fastest
 * per chain.  cache_path (or NULL): buckets found there are not re-timed; the
 * file is rewritten with every bucket's choice (JSON).  SYNCHRONOUS; results
 * of later steps do not depend on the shapes chosen. */
rtt_status rtt_batch_tune(rtt_batch b, const char *cache_path, int32_t probe_chains, void *stream);
/* tile shape currently used for instance i */
rtt_status rtt_batch_shape(rtt_batch b, int32_t instance, int32_t *lanes, int32_t *chains_per_item);

/* ---------------------------------------------------------------------------
 * Learned independence proposal.  A MADE (masked autoregressive MLP, Germain et
 * al. 2015) with two ReLU hidden layers of width H models q(s) as a product of
 * conditionals q(s_order[d] | s_order[<d]) = sigmoid(logit_d); it is trained by
 * this library's kernels (FP32) on configurations the RTT chains produce and
 * proposes s' ~ q for an independence Metropolis-Hastings step on
 * P = |psi|^2/Z (Sec. 3.3): accept iff log u < 2(log|psi(s')| - log|psi(s)|)
 * + log q(s) - log q(s').  The exact RTT ratio decides every acceptance.
 *   Parameters are flat FP32 in the order W1 [H][N], b1 [H], W2 [H][H], b2 [H],
 * W3 [N][H], b3 [N]; masks keep W1[k][d] iff m_k >= d+1, W2[k2][k1] iff
 * m_k2 >= m_k1, W3[d][k] iff d+1 > m_k, with hidden degrees m_k = (k mod
 * (N-1)) + 1.  Random bits come from Philox4x64-10 with key (seed, 0x4D414445)
 * and counter (chain, round, position d) for the sample bits, position N for
 * the acceptance uniform.  The paper's method has no learned proposal; this is
 * the sampler extension the hot path carries beside local flips.
 * --------------------------------------------------------------------------- */
typedef struct rtt_made_s *rtt_made;
/* order: host [N] permutation (position -> spin); init_weights: host flat
 * double [P] (masked on load); seed keys the sampling stream. */
rtt_status rtt_made_create(int32_t n_spins, int32_t hidden, const int32_t *order,
                           const double *init_weights, uint64_t seed, int32_t device, rtt_made *out);
rtt_status rtt_made_destroy(rtt_made m);
/* parameters to host float [P] (SYNCHRONOUS) */
rtt_status rtt_made_get_params(rtt_made m, float *host_out);
/* mean NLL gradient of a batch of spins (device [B][N]) into grads (device
 * float [P]); nll (device double, or NULL) receives the mean NLL. */
rtt_status rtt_made_gradients(rtt_made m, const uint8_t *spins, int64_t B, float *grads,
                              double *nll, void *stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean NLL of a batch */
rtt_status rtt_made_train_step(rtt_made m, const uint8_t *spins, int64_t B, float lr, double *nll,
                               void *stream);
/* Minibatch training: `epochs` passes over data (device uint8 [n][N]); each
 * pass visits the rows in a keyed random order (rtt_made_permutation with
 * shuffle_seed and the pass number) in n / batch minibatches of `batch`
 * rows (the last n mod batch rows of each order are skipped), one Adam step
 * per minibatch as rtt_made_train_step.  The rows are gathered on the device;
 * data must stay valid until the stream reaches the end of the call's work.
 * nll_per_epoch: host double [epochs] (mean over the pass's minibatches of
 * their mean NLL) or NULL; when given, the call waits for the stream before it
 * returns.  Errors: RTT_ERR_INVALID_ARG for n < 1, batch outside [1, n],
 * epochs < 0 or lr <= 0 (nothing launched); RTT_ERR_OOM / RTT_ERR_CUDA. */
rtt_status rtt_made_fit(rtt_made m, const uint8_t *data, int64_t n, int32_t epochs, int32_t batch,
                        float lr, uint64_t shuffle_seed, double *nll_per_epoch, void *stream);
/* The training loop's row order for one pass: host_out[i] (host int64 [n]) is
 * the data row visited i-th.  A permutation of [0, n): a four-round Feistel
 * network over [0, 4^h), 4^h >= n, keyed by (seed, epoch), restricted to
 * [0, n) by cycle walking.  Host only; RTT_ERR_INVALID_ARG for n < 1. */
rtt_status rtt_made_permutation(int64_t n, uint64_t seed, int64_t epoch, int64_t *host_out);
/* Inference arithmetic of the H x H layer (sampling, log q, the independence
 * step): bf16 = 1 runs it on the tensor cores -- ReLU(first layer) and the
 * masked W2 rounded to BF16, FP32 accumulation, the same kernel for sampling
 * and for evaluation, so the density a proposal is drawn from is exactly the
 * one the acceptance test evaluates; bf16 = 0 runs it in FP32 on the CUDA
 * cores.  Training is set apart (rtt_made_set_training).  BF16 needs H in {64, 128, 192, 256,
 * 512} (RTT_ERR_UNSUPPORTED otherwise) and is the default for those. */
rtt_status rtt_made_set_inference(rtt_made m, int32_t bf16);
/* Arithmetic of the training GEMMs (forward and backward of rtt_made_gradients,
 * rtt_made_train_step and rtt_made_fit): tc = 1 runs them on the tensor
 * cores, each FP32 operand split into BF16 hi + lo and three products hi.hi +
 * hi.lo + lo.hi accumulated in FP32 (relative error O(2^-16) per product);
 * tc = 0 (the default: faster at the model sizes the sampler trains, whose
 * 128 x 128 output tiles leave most SMs idle) runs them in FP32 on the CUDA
 * cores (FMA in increasing k).
 * Host only, no device work; RTT_ERR_INVALID_ARG for a null model.  A bounded
 * wait that runs out in the tensor-core GEMM sets bit 0 of the flags that
 * rtt_made_device_status reports. */
rtt_status rtt_made_set_training(rtt_made m, int32_t tc);
/* Device-side error flags of the model's tensor-core layer since the last
 * call (bit 0: a bounded wait ran out of its clock budget; that CTA recorded
 * the flag, drained its own copies, freed its tensor memory and returned
 * without writing its rows).  SYNCHRONOUS; RTT_ERR_TIMEOUT if bit 0 is set;
 * clears the flags.  flags: host int32 or NULL. */
rtt_status rtt_made_device_status(rtt_made m, int32_t *flags);
/* log q(s) for B configurations: logq device double [B] */
rtt_status rtt_made_log_prob(rtt_made m, const uint8_t *spins, int64_t B, double *logq, void *stream);
/* B samples s' ~ q (device [B][N]) with their log q (device [B]) */
rtt_status rtt_made_sample(rtt_made m, int64_t B, int64_t chain0, int64_t round, uint8_t *spins,
                           double *logq, void *stream);
/* One independence proposal per chain: s' ~ q, psi(s') by the handle's
 * precision, accept/reject as above; spins and state updated in place,
 * n_accept (device [B] or NULL) counts acceptances. */
rtt_status rtt_indep_mh(rtt_handle h, rtt_made m, uint8_t *spins, rtt_chain_state *state,
                        int64_t B, int64_t chain0, int64_t round, int64_t *n_accept, void *stream);

/* ---------------------------------------------------------------------------
 * Replica-space optimization (Sec. 3.1; rules of Sec. 2.2.3)
 *
 * phi is a TT over the replica space: L sites i_1..i_L in {0,1},
 * phi_i = G_1[i_1] G_2[i_2] ... G_L[i_L] with open ends.  Storage ("padded
 * cores"): device double [L][2][chi][chi], element [k][s][a][b] = G_k[a,s,b];
 * the first core uses row 0 only, the last core column 0 only, and all other
 * entries beyond a bond's rank are zero.  The RTT psi = C phi (Eq.
 * rtt_equal_C_tt) is the handle of rtt_create with these tensors, the same
 * path and b_L = b_R = e_0.
 *
 * A replica-space Pauli string is one code per site: 0 identity, 1 X, 2 Z
 * (uint8).  Applied to a TT it is a rank-1 MPO: X swaps a core's two
 * physical slices, Z negates slice 1.
 * ------------------------------------------------------------------------- */

/* Lift physical Pauli terms to replica-space strings by the commutation rules
 * of Sec. 2.2.3: Z_j is sent to one replica of spin j (the term's block), X_j
 * becomes X on every replica of j.  The path must be a concatenation of
 * orderings, each a permutation of the n_spins spins (block c = sites
 * [c n_spins, (c+1) n_spins)).  Term k has coefficient coef[k], block
 * block[k], and factors offsets[k]..offsets[k+1]-1 of (spins, ops) with ops
 * 1 = X, 2 = Z (3 = Y is rejected: it would make the TT complex); a term may
 * not name a spin twice.  Outputs: ops_out [n_terms][length] string codes and
 * eta_out [n_terms] (= coef).  All pointers host; no device work, callable
 * without a GPU.  RTT_ERR_INVALID_ARG on a malformed path or term,
 * RTT_ERR_UNSUPPORTED for Y. */
rtt_status rtt_replica_lift(int32_t n_spins, int32_t length, const int32_t *path, int32_t n_terms,
                            const double *coef, const int32_t *block, const int32_t *offsets,
                            const int32_t *spins, const uint8_t *ops, uint8_t *ops_out,
                            double *eta_out);

typedef struct rtt_tt_plan_s *rtt_tt_plan;

/* A plan for (1 - tau H-bar) on TTs of `length` sites and rank chi (1..16),
 * H-bar = sum_k eta[k] P_k with the strings ops [n_terms][length] (host,
 * codes as above; n_terms >= 1, length >= 2).  chi_tree: the rank the tree's
 * pairwise sums are rounded to (chi <= chi_tree <= 16; 0 = min(2 chi, 16),
 * the rank a sum of two rank-chi TTs has); the final results (phi, operator
 * states, combinations) are rounded to chi.  precision: RTT_FP64 or
 * RTT_FP32, the arithmetic of the roundings (cores are FP64 in memory either
 * way; FP32 runs the factorizations at the FP32 rate, with correspondingly
 * larger rounding errors).  Copies the strings to the device, allocates the
 * tree's node TTs (n_terms - 1 of them, rank chi_tree) and the rounding
 * scratch (floor(n_terms/2) * length * 2 * (2 c)^2 values, c = max(chi,
 * chi_tree) rounded up to 2, 4, 8 or 16) on `device`.  *out owned by the
 * caller (rtt_tt_plan_destroy). */
rtt_status rtt_tt_plan_create(int32_t length, int32_t chi, int32_t chi_tree, int32_t precision,
                              int32_t n_terms, const uint8_t *ops, const double *eta,
                              int32_t device, rtt_tt_plan *out);
rtt_status rtt_tt_plan_destroy(rtt_tt_plan plan);

/* n_steps applications of 1 - tau H-bar to phi in place (device padded
 * cores), each as Sec. 3.1 orders it: the terms eta_k P_k phi, summed two by
 * two (items in term order; pairs (0,1), (2,3), ...; an odd last item passes
 * to the next level unchanged) with every pair sum rounded to rank chi, until
 * one TT S is left (pairwise sums rounded to chi_tree); then
 * phi <- round(phi - tau S) / ||.||_2 at rank chi.  Rounding is
 * TT rounding: left-to-right Householder QR of each core, then right-to-left
 * SVD (one-sided Jacobi) keeping the chi largest singular values per bond.
 * The output's cores 2..L are right-orthonormal and core 1 carries the
 * replica-space norm, which is scaled to 1; log_norm (device double
 * [n_steps] or NULL) receives log ||round(phi - tau S)||_2 of every step (a
 * non-finite entry means the step failed numerically).  One kernel launch
 * per tree level and one for the final sum per step, plus one
 * device-to-device copy; ordered on `stream`.  RTT_ERR_INVALID_ARG for a null
 * phi or n_steps < 0. */
rtt_status rtt_tt_power(rtt_tt_plan plan, double *phi, double tau, int32_t n_steps,
                        double *log_norm, void *stream);

/* phi^alpha = O-bar phi for the plan's operator O-bar = sum_k eta[k] P_k
 * (Sec. 3.2: psi^alpha = O_alpha psi built with the lifted operator as in the
 * replica-space optimization): the terms eta_k P_k phi summed two by two with
 * a rounding to chi_tree after every sum, the root rounded to the plan's chi
 * and scaled to unit norm; log_norm (device double [1] or NULL) receives the
 * log of the norm before scaling.  phi: device padded cores of rank chi_phi
 * (0 = the plan's chi; at most max(chi, chi_tree)); out: the plan's chi; out
 * must not alias phi.  Uses the plan's node buffers and scratch (calls on one
 * plan are ordered by the caller).  One launch per tree level plus one. */
rtt_status rtt_tt_apply(rtt_tt_plan plan, const double *phi, int32_t chi_phi, double *out,
                        double *log_norm, void *stream);

/* out = round(sum_m coef[m] tts[m]) scaled to unit norm (Eq. lin_comb: the
 * optimal combination turned back into one TT), the sum taken two by two with
 * a rounding to chi_tree after every sum and the root rounded to chi, like
 * rtt_tt_apply.  n <= the plan's n_terms (the plan's node buffers hold the
 * tree); tts: host array of n device padded-core pointers of the plan's
 * length and rank chi_in (0 = chi; at most max(chi, chi_tree)); coef: host
 * [n]; out: the plan's chi; log_norm as above. */
rtt_status rtt_tt_sum_round(rtt_tt_plan plan, int32_t n, const double *const *tts, int32_t chi_in,
                            const double *coef, double *out, double *log_norm, void *stream);

/* One rounding of a two-term sum, the operation every tree node performs:
 * out = round(coef_a P_a a + coef_b P_b b) (device padded cores, each of the
 * plan's length and chi; ops_a / ops_b device string rows [length] or NULL
 * for the identity).  If log_norm (device double [1]) is not NULL the result
 * is scaled to unit norm and the log of its norm stored there.  out must not
 * alias a or b.  Uses the plan's scratch: calls on one plan are ordered on
 * their streams by the caller. */
rtt_status rtt_tt_round_sum(rtt_tt_plan plan, const double *a, const uint8_t *ops_a, double coef_a,
                            const double *b, const uint8_t *ops_b, double coef_b, double *out,
                            double *log_norm, void *stream);

/* The local energy of rtt_local_energy (same kernels, same results) from a
 * call that allocates no device memory.  The paper has no counterpart: this
 * is an operational variant for callers that cannot allocate at the time of
 * the call -- loops that forbid allocator calls after start-up, or programs
 * whose device memory is owned by an external pool manager that must make
 * every allocation itself.
 *   Scratch comes from one 32 MiB array compiled into the library as a device
 * global (every GPU that loads the library holds it until the process exits);
 * a batch whose scratch -- two stacks of B*N*chi_p values (8 B in FP64, 4 B in
 * FP32) plus 4 B exponents each, and 16 B * B*(N+1) for the rows -- exceeds
 * 32 MiB is rejected with RTT_ERR_INVALID_ARG before anything is launched
 * (split the batch).  FP64 and FP32 handles only (RTT_ERR_UNSUPPORTED else).
 *   The first call on a device looks up the array's device address with that
 * device current (once per device); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents:
 * nothing needs clearing (every entry is written before it is read), but
 * calls that overlap on the GPU -- on different streams, or from threads
 * without ordering -- race on it; serialize them.  spins, e_loc, ratios and
 * stream as for rtt_local_energy. */
rtt_status rtt_local_energy_noalloc(rtt_handle h, const uint8_t *spins, int64_t B,
                                    double *e_loc, double *ratios, void *stream);

/* Device-side error flags of the handle's kernels since the last call
 * (bit 0: a bounded wait inside a tensor-core kernel ran out of its clock
 * budget; that kernel recorded the flag, drained its own copies, freed its
 * tensor memory and returned without writing results).  SYNCHRONOUS.
 * Returns RTT_ERR_TIMEOUT if bit 0 is set, and clears the flags. */
rtt_status rtt_device_status(rtt_handle h, int32_t *flags);
/* Failure-detection self-test (no counterpart in the paper: it exercises the
 * path a tensor-core kernel takes when one of its bounded waits runs out).
 * One warp arms an mbarrier that no copy and no MMA will ever arrive on and
 * waits on it with a clock budget of budget_cycles; when the budget runs out
 * it records bit 0 in the handle's device error word, frees the tensor memory
 * it holds and returns.  Nothing asynchronous is in flight when it gives up,
 * so the context stays usable: the next rtt_device_status returns
 * RTT_ERR_TIMEOUT (and clears the flag) and later calls on the handle run
 * normally.  budget_cycles in [1e3, 4e9] (SM clock cycles; 2e6 is about 1 ms)
 * else RTT_ERR_INVALID_ARG; BF16X3 / FP16X3 handles only (RTT_ERR_UNSUPPORTED
 * otherwise).  Asynchronous on `stream`. */
rtt_status rtt_wait_selftest(rtt_handle h, int64_t budget_cycles, void *stream);

/* Bytes of device scratch a handle holds for batches of B chains. */
rtt_status rtt_scratch_bytes(rtt_handle h, int64_t B, size_t *bytes);

const char *rtt_status_string(rtt_status s);
const char *rtt_last_error(void);   /* thread-local; "" when none */

#ifdef __cplusplus
}
#endif
#endif /* RTT_H */
