/*
 * rtt_oracle.c -- plain, slow, FP64 CPU reference of the RTT Monte Carlo hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - RTT amplitude psi_s = Tr A_1^{s_sigma(1)} ... A_Omega^{s_sigma(Omega)}
 *     (Sec. 2.2.1, Eq. RTT), with the first/last bond of dimension one
 *     (Sec. 2.1) realised as boundary vectors b_L, b_R.
 *   - single-flip amplitudes psi(s^(i)) by the factorisation
 *     l_{a-1} . A_a ... A_b . r_{b+1}, a/b the first/last train site of spin i
 *     (replica set R_i, Sec. 2.2.1), with l and r rebuilt from scratch for
 *     every flip.
 *   - the TFIM local energy E_loc(s) = sum_sbar H_{s,sbar} psi_sbar / psi_s
 *     (Sec. 3.3, the mixed local energy with psi^1 = psi^2; Hamiltonian of
 *     Sec. 4, Eq. ising-model) with J sum z_i z_j - h sum X_i.
 *   - Metropolis sampling of P_s = |psi_s|^2 / Z (Sec. 3.3) by systematic
 *     single-spin sweeps; uniforms from Philox4x64-10 (Salmon et al., SC'11).
 *   - exact <H> by enumerating all 2^N configurations (N <= 20).
 *   - the mixed local energy and overlap ratio of dual Monte Carlo (Sec. 3.3)
 *     between two RTTs on the same lattice.
 *
 * Arithmetic conventions (the canonical order the FP64 GPU path reproduces):
 *   - vector x matrix: out[b] = sum_a v[a] A[a][b], accumulated with fma()
 *     from +0 in increasing a; matrix x vector: out[a] = sum_b A[a][b] r[b],
 *     fma in increasing b; dot products likewise in increasing index.
 *   - after every site the vector is scaled by 2^-e with e = ilogb(max|v|),
 *     which is exact; the exponents are summed in an int64.
 *   - spin encoding s = 0 <-> z = +1, s = 1 <-> z = -1.
 *
 * Compile with -ffp-contract=off (no implicit fma contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n_spins;       /* N                                   */
    int32_t length;        /* L = number of train sites (Omega)   */
    int32_t chi;           /* uniform bond dimension              */
    int32_t n_bonds;
    const int32_t *path;   /* [L]  sigma(k) in [0, N)             */
    const double *tensors; /* [L][2][chi][chi]  A_k[s][a][b]      */
    const double *b_left;  /* [chi]                                */
    const double *b_right; /* [chi]                                */
    const int32_t *bonds;  /* [n_bonds][2]                         */
    double J, h;
} orc_rtt;

/* ---------------------------------------------------------------- helpers */

static const double *site_matrix(const orc_rtt *m, int k, int s)
{
    return m->tensors + ((size_t)k * 2 + (size_t)s) * (size_t)m->chi * (size_t)m->chi;
}

/* Scale v by a power of two so that max|v| lies in [1, 2); return the exponent. */
static int64_t renorm(double *v, int chi)
{
    double mx = 0.0;
    for (int b = 0; b < chi; ++b) {
        double a = fabs(v[b]);
        if (a > mx) mx = a;
    }
    if (mx == 0.0 || !isfinite(mx)) return 0;
    int e = ilogb(mx);
    for (int b = 0; b < chi; ++b) v[b] = ldexp(v[b], -e);
    return (int64_t)e;
}

/* out = v . A_k[s]  (row vector times matrix) */
static void step_left(const orc_rtt *m, int k, int s, const double *v, double *out)
{
    const int chi = m->chi;
    const double *A = site_matrix(m, k, s);
    for (int b = 0; b < chi; ++b) {
        double acc = 0.0;
        for (int a = 0; a < chi; ++a) acc = fma(v[a], A[(size_t)a * chi + b], acc);
        out[b] = acc;
    }
}

/* out = A_k[s] . r  (matrix times column vector) */
static void step_right(const orc_rtt *m, int k, int s, const double *r, double *out)
{
    const int chi = m->chi;
    const double *A = site_matrix(m, k, s);
    for (int a = 0; a < chi; ++a) {
        double acc = 0.0;
        for (int b = 0; b < chi; ++b) acc = fma(A[(size_t)a * chi + b], r[b], acc);
        out[a] = acc;
    }
}

static double dot(const double *u, const double *r, int chi)
{
    double acc = 0.0;
    for (int b = 0; b < chi; ++b) acc = fma(u[b], r[b], acc);
    return acc;
}

/* Bring a scalar mantissa into [1,2) in magnitude (exact). */
static void normalize_scalar(double *mant, int64_t *ex)
{
    if (*mant == 0.0 || !isfinite(*mant)) return;
    int e = ilogb(*mant);
    *mant = ldexp(*mant, -e);
    *ex += e;
}

/* ---------------------------------------------------------------- amplitude */

/* psi(s) = b_L^T A_0[s_p(0)] ... A_{L-1}[s_p(L-1)] b_R, left to right.
 * Result psi = mant * 2^ex with |mant| in [1,2) (or mant == 0). */
void orc_amplitude(const orc_rtt *m, const uint8_t *s, double *mant, int64_t *ex)
{
    const int chi = m->chi;
    double *v = (double *)malloc(sizeof(double) * chi);
    double *w = (double *)malloc(sizeof(double) * chi);
    memcpy(v, m->b_left, sizeof(double) * chi);
    int64_t E = 0;
    for (int k = 0; k < m->length; ++k) {
        step_left(m, k, s[m->path[k]], v, w);
        double *t = v; v = w; w = t;
        E += renorm(v, chi);
    }
    double mm = dot(v, m->b_right, chi);
    normalize_scalar(&mm, &E);
    *mant = mm;
    *ex = E;
    free(v);
    free(w);
}

/* Amplitude of s with spin `flip` inverted (flip < 0: no flip), by the
 * factorisation l_{a-1} . (A_a ... A_b) . r_{b+1} where a, b are the first and
 * last train sites carrying that spin; l and r are rebuilt from scratch. */
void orc_flip_amplitude(const orc_rtt *m, const uint8_t *s, int flip,
                        double *mant, int64_t *ex)
{
    if (flip < 0) {
        orc_amplitude(m, s, mant, ex);
        return;
    }
    const int chi = m->chi, L = m->length;
    int a = -1, b = -1;
    for (int k = 0; k < L; ++k)
        if (m->path[k] == flip) {
            if (a < 0) a = k;
            b = k;
        }
    double *l = (double *)malloc(sizeof(double) * chi);
    double *r = (double *)malloc(sizeof(double) * chi);
    double *w = (double *)malloc(sizeof(double) * chi);
    /* left environment l_{a-1} */
    memcpy(l, m->b_left, sizeof(double) * chi);
    int64_t El = 0;
    for (int k = 0; k < a; ++k) {
        step_left(m, k, s[m->path[k]], l, w);
        double *t = l; l = w; w = t;
        El += renorm(l, chi);
    }
    /* right environment r_{b+1} */
    memcpy(r, m->b_right, sizeof(double) * chi);
    int64_t Er = 0;
    for (int k = L - 1; k > b; --k) {
        step_right(m, k, s[m->path[k]], r, w);
        double *t = r; r = w; w = t;
        Er += renorm(r, chi);
    }
    /* flipped segment a..b */
    for (int k = a; k <= b; ++k) {
        int p = m->path[k];
        int sk = s[p] ^ (p == flip ? 1 : 0);
        step_left(m, k, sk, l, w);
        double *t = l; l = w; w = t;
        El += renorm(l, chi);
    }
    double mm = dot(l, r, chi);
    int64_t E = El + Er;
    normalize_scalar(&mm, &E);
    *mant = mm;
    *ex = E;
    free(l);
    free(r);
    free(w);
}

/* Conditioning of the left-to-right evaluation of psi(s), for stating
 * floating-point tolerances: for every site kappa_k = || |v| |A_k| ||_2 /
 * || v A_k ||_2 (v the incoming row, |.| elementwise), and for the closing
 * contraction kappa_fin = sum_b |v_b b_R[b]| / |sum_b v_b b_R[b]|.  Returns
 * sum_k kappa_k in *sum_kappa, max_k kappa_k in *max_kappa and kappa_fin. */
void orc_amplitude_cond(const orc_rtt *m, const uint8_t *s, double *sum_kappa,
                        double *max_kappa, double *kappa_fin)
{
    const int chi = m->chi;
    double *v = (double *)malloc(sizeof(double) * chi);
    double *w = (double *)malloc(sizeof(double) * chi);
    memcpy(v, m->b_left, sizeof(double) * chi);
    double sk = 0.0, mk = 0.0;
    for (int k = 0; k < m->length; ++k) {
        const double *A = site_matrix(m, k, s[m->path[k]]);
        double num = 0.0, den = 0.0;
        for (int b = 0; b < chi; ++b) {
            double acc = 0.0, aacc = 0.0;
            for (int a = 0; a < chi; ++a) {
                acc = fma(v[a], A[(size_t)a * chi + b], acc);
                aacc += fabs(v[a]) * fabs(A[(size_t)a * chi + b]);
            }
            w[b] = acc;
            num += aacc * aacc;
            den += acc * acc;
        }
        double kap = (den > 0.0) ? sqrt(num / den) : INFINITY;
        sk += kap;
        if (kap > mk) mk = kap;
        double *t = v; v = w; w = t;
        renorm(v, chi);
    }
    double num = 0.0, den = 0.0;
    for (int b = 0; b < chi; ++b) {
        num += fabs(v[b] * m->b_right[b]);
        den = fma(v[b], m->b_right[b], den);
    }
    *sum_kappa = sk;
    *max_kappa = mk;
    *kappa_fin = (den != 0.0) ? num / fabs(den) : INFINITY;
    free(v);
    free(w);
}

/* ---------------------------------------------------------------- energy */

static int64_t zz_sum(const orc_rtt *m, const uint8_t *s)
{
    int64_t zz = 0;
    for (int q = 0; q < m->n_bonds; ++q) {
        int i = m->bonds[2 * q], j = m->bonds[2 * q + 1];
        int zi = 1 - 2 * (int)s[i], zj = 1 - 2 * (int)s[j];
        zz += (int64_t)(zi * zj);
    }
    return zz;
}

/* E_loc(s) = J sum_<ij> z_i z_j - h sum_i psi(s^(i)) / psi(s).
 * ratios (may be NULL) receives psi(s^(i))/psi(s) indexed by spin i.
 * Returns 0, or 1 if psi(s) == 0 (E_loc undefined, set to NaN). */
int orc_local_energy(const orc_rtt *m, const uint8_t *s, double *eloc, double *ratios)
{
    double m0;
    int64_t e0;
    orc_amplitude(m, s, &m0, &e0);
    if (m0 == 0.0 || !isfinite(m0)) {
        *eloc = NAN;
        return 1;
    }
    double sum = 0.0;
    for (int i = 0; i < m->n_spins; ++i) {
        double mi;
        int64_t ei;
        orc_flip_amplitude(m, s, i, &mi, &ei);
        double q = mi / m0;
        double ratio = ldexp(q, (int)(ei - e0));
        if (ratios) ratios[i] = ratio;
        sum += ratio;
    }
    double zz = (double)zz_sum(m, s);
    *eloc = m->J * zz - m->h * sum;
    return 0;
}

/* ---------------------------------------------------------------- Philox4x64-10 */

/* Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten
 * rounds of two 64x64->128 multiplications per round on a 4x64 counter,
 * key schedule bumped by the Weyl constants between rounds. */
static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    __uint128_t p = (__uint128_t)a * (__uint128_t)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t h0, l0, h1, l1;
        mul128(M0, x0, &h0, &l0);
        mul128(M1, x2, &h1, &l1);
        uint64_t y0 = h1 ^ x1 ^ k0;
        uint64_t y1 = l1;
        uint64_t y2 = h0 ^ x3 ^ k1;
        uint64_t y3 = l0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Metropolis uniform for (chain, sweep, proposal): key = (seed, 0x4D434D43),
 * counter = (chain, sweep, proposal, 0); u = (x0 >> 11) * 2^-53 in [0, 1). */
double orc_mcmc_uniform(uint64_t seed, uint64_t chain, uint64_t sweep, uint64_t proposal)
{
    uint64_t ctr[4] = {chain, sweep, proposal, 0};
    uint64_t key[2] = {seed, 0x4D434D43ULL};
    uint64_t x[4];
    orc_philox4x64(ctr, key, x);
    return (double)(x[0] >> 11) * 0x1.0p-53;
}

/* Uniform of an arbitrary keyed stream: key = (seed, stream), counter =
 * (c0, c1, c2, 0); u = (x0 >> 11) * 2^-53.  The learned proposal draws its
 * bits with stream 0x4D414445 ("MADE"), counter (chain, round, position) and
 * its acceptance uniform at position N. */
double orc_uniform_keyed(uint64_t seed, uint64_t stream, uint64_t c0, uint64_t c1, uint64_t c2)
{
    uint64_t ctr[4] = {c0, c1, c2, 0};
    uint64_t key[2] = {seed, stream};
    uint64_t x[4];
    orc_philox4x64(ctr, key, x);
    return (double)(x[0] >> 11) * 0x1.0p-53;
}

/* ---------------------------------------------------------------- Metropolis */

/* Systematic single-spin Metropolis on P_s = |psi_s|^2 / Z.
 * One sweep = N proposals; proposal j flips spin path[j] (the order of the
 * first N train sites, which must visit every spin once).  Acceptance:
 * u < (psi(s')/psi(s))^2, strict.  On acceptance the chain amplitude becomes
 * the flipped amplitude as computed by orc_flip_amplitude.
 *
 * spins   [B][N] in/out;  mant/ex [B] in/out: psi = mant * 2^ex of the
 * current state;  trace [n_meas][B] (may be NULL), n_meas = n_sweeps /
 * measure_every: trace[g] is E_loc of the configuration that enters sweep
 * g * measure_every of this call (each measured iteration evaluates the
 * configuration it starts from, then runs its measure_every sweeps; trailing
 * sweeps beyond n_meas * measure_every are not measured);  n_accept [B]
 * accumulates accepted proposals.
 * Chains are numbered chain0 + c for the random stream.  Returns the number
 * of chains whose amplitude or local energy was undefined. */
int orc_mcmc(const orc_rtt *m, uint64_t seed, uint8_t *spins, double *mant, int64_t *ex,
             int64_t B, int64_t chain0, int64_t sweep0, int32_t n_sweeps,
             int32_t measure_every, double *trace, int64_t *n_accept)
{
    const int N = m->n_spins;
    int bad = 0;
    for (int64_t c = 0; c < B; ++c) {
        uint8_t *s = spins + (size_t)c * N;
        const int32_t n_meas = (trace && measure_every > 0) ? n_sweeps / measure_every : 0;
        int32_t meas = 0;
        for (int32_t t = 0; t < n_sweeps; ++t) {
            int64_t sweep = sweep0 + t;
            if (meas < n_meas && (t % measure_every) == 0) {
                double e;
                bad += orc_local_energy(m, s, &e, NULL);
                trace[(size_t)meas * B + c] = e;
                ++meas;
            }
            for (int j = 0; j < N; ++j) {
                int i = m->path[j];
                double mf;
                int64_t ef;
                orc_flip_amplitude(m, s, i, &mf, &ef);
                double q = mf / mant[c];
                double ratio = ldexp(q, (int)(ef - ex[c]));
                double u = orc_mcmc_uniform(seed, (uint64_t)(chain0 + c), (uint64_t)sweep, (uint64_t)j);
                if (u < ratio * ratio) {
                    s[i] ^= 1;
                    mant[c] = mf;
                    ex[c] = ef;
                    if (n_accept) n_accept[c] += 1;
                }
            }
        }
    }
    return bad;
}

/* ---------------------------------------------------------------- enumeration */

/* Configuration index -> spins: bit (N-1-i) of idx is s_i (spin 0 is the most
 * significant bit, the Kronecker-product order). */
static void index_to_spins(uint64_t idx, int N, uint8_t *s)
{
    for (int i = 0; i < N; ++i) s[i] = (uint8_t)((idx >> (N - 1 - i)) & 1u);
}

/* psi(s) for all 2^N configurations as doubles (ldexp of mant/exponent);
 * psi_out [2^N].  The caller checks that no entry over/underflowed. */
void orc_all_amplitudes(const orc_rtt *m, double *psi_out)
{
    const int N = m->n_spins;
    uint8_t *s = (uint8_t *)malloc((size_t)N);
    for (uint64_t idx = 0; idx < (1ULL << N); ++idx) {
        index_to_spins(idx, N, s);
        double mm;
        int64_t e;
        orc_amplitude(m, s, &mm, &e);
        psi_out[idx] = ldexp(mm, (int)e);
    }
    free(s);
}

/* Exact <psi|H|psi>/<psi|psi> by enumeration (N <= 20):
 * (H psi)(s) = J zz(s) psi(s) - h sum_i psi(s^(i)).  psi is rescaled by its
 * largest entry before forming products.  Returns the energy. */
double orc_exact_energy(const orc_rtt *m, double *norm_out)
{
    const int N = m->n_spins;
    const uint64_t D = 1ULL << N;
    double *psi = (double *)malloc(sizeof(double) * D);
    uint8_t *s = (uint8_t *)malloc((size_t)N);
    orc_all_amplitudes(m, psi);
    double mx = 0.0;
    for (uint64_t idx = 0; idx < D; ++idx)
        if (fabs(psi[idx]) > mx) mx = fabs(psi[idx]);
    for (uint64_t idx = 0; idx < D; ++idx) psi[idx] /= mx;
    double num = 0.0, den = 0.0;
    for (uint64_t idx = 0; idx < D; ++idx) {
        index_to_spins(idx, N, s);
        double hpsi = m->J * (double)zz_sum(m, s) * psi[idx];
        for (int i = 0; i < N; ++i) hpsi -= m->h * psi[idx ^ (1ULL << (N - 1 - i))];
        num += psi[idx] * hpsi;
        den += psi[idx] * psi[idx];
    }
    if (norm_out) *norm_out = den;
    free(psi);
    free(s);
    return num / den;
}

/* ---------------------------------------------------------------- batch helpers */

/* log|psi| and sign for B configurations. */
void orc_log_amplitudes(const orc_rtt *m, const uint8_t *spins, int64_t B,
                        double *log_abs, int8_t *sign, double *mant, int64_t *ex)
{
    const int N = m->n_spins;
    for (int64_t c = 0; c < B; ++c) {
        double mm;
        int64_t e;
        orc_amplitude(m, spins + (size_t)c * N, &mm, &e);
        if (mant) mant[c] = mm;
        if (ex) ex[c] = e;
        if (mm == 0.0) {
            log_abs[c] = -INFINITY;
            sign[c] = 0;
        } else {
            log_abs[c] = (double)e * 0.69314718055994530942 + log(fabs(mm));
            sign[c] = mm > 0 ? 1 : -1;
        }
    }
}

/* E_loc and (optionally) all ratios [B][N] for B configurations. */
int orc_local_energies(const orc_rtt *m, const uint8_t *spins, int64_t B,
                       double *eloc, double *ratios)
{
    const int N = m->n_spins;
    int bad = 0;
    for (int64_t c = 0; c < B; ++c)
        bad += orc_local_energy(m, spins + (size_t)c * N, eloc + c,
                                ratios ? ratios + (size_t)c * N : NULL);
    return bad;
}

/* Single-flip amplitudes for all spins of B configurations: [B][N]. */
void orc_flip_amplitudes(const orc_rtt *m, const uint8_t *spins, int64_t B,
                         double *mant, int64_t *ex)
{
    const int N = m->n_spins;
    for (int64_t c = 0; c < B; ++c)
        for (int i = 0; i < N; ++i)
            orc_flip_amplitude(m, spins + (size_t)c * N, i, mant + (size_t)c * N + i,
                               ex + (size_t)c * N + i);
}

/* ---------------------------------------------------------------- dual Monte Carlo */

/* Mixed local energy of dual Monte Carlo (Sec. 3.3):
 *   E^{ab}(s) = sum_sbar H_{s,sbar} psi^b_sbar / psi^a_s
 *             = [J sum_<ij> z_i z_j psi^b(s) - h sum_i psi^b(s^(i))] / psi^a(s)
 * (Hamiltonian of Sec. 4 taken from b), and the overlap ratio
 * r^{ab}(s) = psi^b(s) / psi^a(s), whose P^a averages are H~_ab and S~_ab.
 * Every amplitude ratio is ldexp(mant_b / mant_a, ex_b - ex_a); the field term
 * adds the N flip ratios in increasing spin index; E = (J zz) r - h sum.
 * Returns 1, with both outputs NaN, when psi^a(s) is zero or not finite. */
int orc_mixed_local_energy(const orc_rtt *ma, const orc_rtt *mb, const uint8_t *s,
                           double *e_mixed, double *ratio)
{
    double m_a, m_b;
    int64_t e_a, e_b;
    orc_amplitude(ma, s, &m_a, &e_a);
    if (m_a == 0.0 || !isfinite(m_a)) {
        *e_mixed = NAN;
        *ratio = NAN;
        return 1;
    }
    orc_amplitude(mb, s, &m_b, &e_b);
    const double r0 = ldexp(m_b / m_a, (int)(e_b - e_a));
    double sum = 0.0;
    for (int i = 0; i < mb->n_spins; ++i) {
        double mi;
        int64_t ei;
        orc_flip_amplitude(mb, s, i, &mi, &ei);
        sum += ldexp(mi / m_a, (int)(ei - e_a));
    }
    const double zz = (double)zz_sum(mb, s);
    *e_mixed = mb->J * zz * r0 - mb->h * sum;
    *ratio = r0;
    return 0;
}

/* The same for B configurations [B][N]; outputs [B]. */
int orc_mixed_local_energies(const orc_rtt *ma, const orc_rtt *mb, const uint8_t *spins,
                             int64_t B, double *e_mixed, double *ratio)
{
    const int N = mb->n_spins;
    int bad = 0;
    for (int64_t c = 0; c < B; ++c)
        bad += orc_mixed_local_energy(ma, mb, spins + (size_t)c * N, e_mixed + c, ratio + c);
    return bad;
}
