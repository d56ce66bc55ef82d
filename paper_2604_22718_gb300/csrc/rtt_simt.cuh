// rtt_simt.cuh -- SIMT (CUDA-core) kernels of the RTT hot path, templated on
// the element type T (double or float) and the padded bond dimension CHI.
//
// Mapping: a "row" (one chi-vector walking along the train) is owned by a
// group of G = min(CHI, 32) lanes of one warp; lane gl of the group owns
// columns gl, gl+G, gl+2G, ...  One site step out = v . A_k[s] (Eq. RTT,
// row vector times matrix) broadcasts v[a] by warp shuffle in increasing a
// and accumulates out[b] with one fma per a -- the same order as the oracle,
// so the FP64 instantiation reproduces it bit for bit.  Right-to-left steps
// use the transposed tensors with the same code.  After every site the row
// is rescaled by 2^-e, e = floor(log2 max|v|) (exact), and e is summed.
//
// Periodic paths (the fast kernels): site k carries spin q[k mod N]; spin
// q[j] lives on sites j, j+N, ..., j+(R-1)N, so its flip touches exactly
// those sites.  General paths (Sec. 2.2.1: the replicas may visit the spins in
// different orders, e.g. sigma^V + sigma^H + sigma^D + sigma^D'): site k
// carries spin p[k]; the first N sites visit every spin once (proposal order);
// spin i's flip touches the sites k with p[k] = i, the last of them last[i].
#pragma once

#include "rtt_internal.cuh"

namespace rttd {

constexpr unsigned FULL = 0xffffffffu;

template <int CHI>
struct Geo {
    static constexpr int G = CHI < 32 ? CHI : 32;   // lanes per row
    static constexpr int NQ = CHI / G;              // columns per lane
    static constexpr int RPW = 32 / G;              // rows per warp
};

// GG lanes per row (default min(CHI, 32)); results do not depend on GG: every
// output column accumulates over a in increasing order whatever the split.
template <typename T, int CHI, int GG = Geo<CHI>::G>
struct RowOps {
    static constexpr int G = GG;
    static constexpr int NQ = CHI / GG;

    // out[b] = sum_a v[a] M[a][b]; M row-major [CHI][CHI].
    static __device__ __forceinline__ void vecmat(const T *__restrict__ M, const T (&v)[NQ],
                                                  T (&out)[NQ], int gl) {
        T acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = T(0);
#pragma unroll
        for (int aq = 0; aq < NQ; ++aq) {
#pragma unroll(G < 8 ? G : 8)
            for (int al = 0; al < G; ++al) {
                const T va = __shfl_sync(FULL, v[aq], al, G);
                const T *row = M + (size_t)(aq * G + al) * CHI + gl;
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc[q] = fma(va, __ldg(row + q * G), acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] = acc[q];
    }

    // Rescale by a power of two so that max|v| is in [1,2); return the exponent.
    static __device__ __forceinline__ int renorm(T (&v)[NQ]) {
        T m = T(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) m = fmax(m, fabs(v[q]));
#pragma unroll
        for (int off = G / 2; off >= 1; off >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, off, G));
        if (!(m > T(0)) || !isfinite(m)) return 0;
        const int e = exponent_of(m);
        if (pow2_normal(T(0), -e)) {  // one exact multiply per entry
            const T sc = pow2(T(0), -e);
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[q] *= sc;
        } else {
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[q] = scale2(v[q], -e);
        }
        return e;
    }

    // sum_b u[b] r[b] accumulated in FP64 (exact products of FP32 inputs; for
    // T = double this is the oracle's fma order), in increasing b; every lane
    // of the group gets it.
    static __device__ __forceinline__ double dot(const T (&u)[NQ], const T (&r)[NQ]) {
        double acc = 0.0;
#pragma unroll
        for (int aq = 0; aq < NQ; ++aq) {
#pragma unroll(G < 8 ? G : 8)
            for (int al = 0; al < G; ++al) {
                const double ua = (double)__shfl_sync(FULL, u[aq], al, G);
                const double ra = (double)__shfl_sync(FULL, r[aq], al, G);
                acc = fma(ua, ra, acc);
            }
        }
        return acc;
    }

    static __device__ __forceinline__ void load(const T *__restrict__ p, T (&v)[NQ], int gl) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = p[gl + q * G];
    }
    static __device__ __forceinline__ void store(T *__restrict__ p, const T (&v)[NQ], int gl) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) p[gl + q * G] = v[q];
    }
};

__device__ __forceinline__ void normalize_scalar(double &m, int64_t &e) {
    if (m == 0.0 || !isfinite(m)) return;
    const int k = exponent_of(m);
    m = scale2(m, -k);
    e += k;
}

template <typename T, int CHI>
__device__ __forceinline__ const T *site(const T *A, int k, int s) {
    return A + ((size_t)k * 2 + (size_t)s) * (size_t)CHI * CHI;
}

struct KArgs {
    const void *A, *AT, *bl, *br;
    const int32_t *q;
    int N, L, R;
    // general paths only (p == nullptr for a periodic path)
    const int32_t *p;     // [L] spin of site k
    const int32_t *last;  // [N] last site of spin i
    int kmin;             // right stack entry e holds r_{kmin+e}; e = L-kmin is b_R
};

// ---------------------------------------------------------------------------
// left environments l_j = b_L A_0 ... A_j (j < N), one group per chain
// ---------------------------------------------------------------------------
template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_left_env(KArgs a, const uint8_t *__restrict__ spins,
                                                  int64_t B, T *__restrict__ lstack,
                                                  int32_t *__restrict__ lexp) {
    using O = RowOps<T, CHI>;
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const bool active = c0 < B;
    const int64_t c = active ? c0 : B - 1;
    const T *A = (const T *)a.A;
    const uint8_t *s = spins + c * a.N;
    T v[O::NQ];
    O::load((const T *)a.bl, v, gl);
    int32_t E = 0;
    for (int j = 0; j < a.N; ++j) {
        const int sp = __ldg(s + __ldg(a.q + j));
        O::vecmat(site<T, CHI>(A, j, sp), v, v, gl);
        E += O::renorm(v);
        if (active) {
            O::store(lstack + ((size_t)c * a.N + j) * CHI, v, gl);
            if (gl == 0) lexp[(size_t)c * a.N + j] = E;
        }
    }
}

// ---------------------------------------------------------------------------
// right environments of the last block: entry q holds r_{(R-1)N+1+q}
// (q = N-1 is b_R itself), one group per chain
// ---------------------------------------------------------------------------
template <typename T, int CHI, int GG = Geo<CHI>::G>
__device__ __forceinline__ void right_env_chain(const KArgs &a, const uint8_t *s, T *rstack_c,
                                                int32_t *rexp_c, bool active, int gl) {
    using O = RowOps<T, CHI, GG>;
    const T *AT = (const T *)a.AT;
    T r[O::NQ];
    O::load((const T *)a.br, r, gl);
    int32_t E = 0;
    const int base = (a.R - 1) * a.N + 1;
    if (active) {
        O::store(rstack_c + (size_t)(a.N - 1) * CHI, r, gl);
        if (gl == 0) rexp_c[a.N - 1] = 0;
    }
    for (int k = a.L - 1; k >= base; --k) {
        const int sp = s[__ldg(a.q + (k % a.N))];
        O::vecmat(site<T, CHI>(AT, k, sp), r, r, gl);
        E += O::renorm(r);
        if (active) {
            O::store(rstack_c + (size_t)(k - base) * CHI, r, gl);
            if (gl == 0) rexp_c[k - base] = E;
        }
    }
}

template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_right_env(KArgs a, const uint8_t *__restrict__ spins,
                                                   int64_t B, T *__restrict__ rstack,
                                                   int32_t *__restrict__ rexp) {
    using O = RowOps<T, CHI>;
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const bool active = c0 < B;
    const int64_t c = active ? c0 : B - 1;
    right_env_chain<T, CHI>(a, spins + c * a.N, rstack + (size_t)c * a.N * CHI,
                            rexp + (size_t)c * a.N, active, gl);
}

// ---------------------------------------------------------------------------
// rows: group (c, j), j in [0, N].  j < N: psi(s^(q[j])) = l_{j-1} .
// A_j[s'] ... A_{(R-1)N+j}[s'] . r_{(R-1)N+j+1};  j = N: psi(s) = l_{N-1} .
// A_N ... A_{L-1} . b_R.
// ---------------------------------------------------------------------------
template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_rows(KArgs a, const uint8_t *__restrict__ spins, int64_t B,
                                              const T *__restrict__ lstack,
                                              const int32_t *__restrict__ lexp,
                                              const T *__restrict__ rstack,
                                              const int32_t *__restrict__ rexp,
                                              double *__restrict__ rows_mant,
                                              int64_t *__restrict__ rows_exp) {
    using O = RowOps<T, CHI>;
    constexpr int RPW = Geo<CHI>::RPW;
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    // group g -> (chain block cb, j, r): the RPW groups of one warp share j
    // (hence the loop length), so the warp's shuffles never diverge.
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const int64_t n_cb = (B + RPW - 1) / RPW;
    const int64_t total = n_cb * (a.N + 1) * RPW;
    const int64_t gg = g0 < total ? g0 : total - 1;
    const int r_in = (int)(gg % RPW);
    const int j = (int)((gg / RPW) % (a.N + 1));
    const int64_t c0 = (gg / RPW / (a.N + 1)) * RPW + r_in;
    const bool active = g0 < total && c0 < B;
    const int64_t c = c0 < B ? c0 : B - 1;
    const int64_t g = c * (a.N + 1) + j;
    const uint8_t *s = spins + c * a.N;
    const T *A = (const T *)a.A;
    T u[O::NQ];
    int64_t E;
    if (j == 0) {
        O::load((const T *)a.bl, u, gl);
        E = 0;
    } else {
        O::load(lstack + ((size_t)c * a.N + (j - 1)) * CHI, u, gl);
        E = lexp[(size_t)c * a.N + (j - 1)];
    }
    const int end = (j < a.N) ? (a.R - 1) * a.N + j : a.L - 1;
    int t = j % a.N;  // k mod N
    for (int k = j; k <= end; ++k) {
        const int sp = __ldg(s + __ldg(a.q + t)) ^ ((t == j) ? 1 : 0);
        O::vecmat(site<T, CHI>(A, k, sp), u, u, gl);
        E += O::renorm(u);
        if (++t == a.N) t = 0;
    }
    const int rq = (j < a.N) ? j : a.N - 1;
    T r[O::NQ];
    O::load(rstack + ((size_t)c * a.N + rq) * CHI, r, gl);
    E += rexp[(size_t)c * a.N + rq];
    double m = O::dot(u, r);
    normalize_scalar(m, E);
    if (active && gl == 0) {
        rows_mant[g] = m;
        rows_exp[g] = E;
    }
}

// ---------------------------------------------------------------------------
// chain init / log amplitudes: full left-to-right pass, one group per chain
// ---------------------------------------------------------------------------
template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_chain_init(KArgs a, const uint8_t *__restrict__ spins,
                                                    int64_t B, double *__restrict__ log_abs,
                                                    int8_t *__restrict__ sign,
                                                    rtt_chain_state *__restrict__ state) {
    using O = RowOps<T, CHI>;
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const bool active = c0 < B;
    const int64_t c = active ? c0 : B - 1;
    const uint8_t *s = spins + c * a.N;
    const T *A = (const T *)a.A;
    T v[O::NQ];
    O::load((const T *)a.bl, v, gl);
    int64_t E = 0;
    int t = 0;
    for (int k = 0; k < a.L; ++k) {
        const int sp = __ldg(s + __ldg(a.p ? a.p + k : a.q + t));
        O::vecmat(site<T, CHI>(A, k, sp), v, v, gl);
        E += O::renorm(v);
        if (++t == a.N) t = 0;
    }
    T r[O::NQ];
    O::load((const T *)a.br, r, gl);
    double m = O::dot(v, r);
    normalize_scalar(m, E);
    if (active && gl == 0) {
        if (state) {
            state[c].mant = m;
            state[c].exp2 = E;
        }
        if (log_abs) log_abs[c] = (m == 0.0) ? -INFINITY : (double)E * 0.6931471805599453 + log(fabs(m));
        if (sign) sign[c] = (m > 0.0) ? 1 : ((m < 0.0) ? -1 : 0);
    }
}

// ---------------------------------------------------------------------------
// Metropolis sweeps, one group per chain (the chain's spins live in shared
// memory).  Per sweep: right environments of the last block from the current
// spins; then for j = 0..N-1 the flipped row from l_{j-1}, both slices of the
// first site (flipped start and unflipped continuation), accept/reject, and
// l_j from the surviving slice.  On the last sweep l_j is stored for the
// local energy that follows.
// ---------------------------------------------------------------------------
template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_sweep(KArgs a, uint8_t *__restrict__ spins,
                                               rtt_chain_state *__restrict__ state, int64_t B,
                                               int64_t chain0, int64_t sweep0, int n_sweeps,
                                               uint64_t seed, T *__restrict__ rstack,
                                               int32_t *__restrict__ rexp, T *__restrict__ lstack,
                                               int32_t *__restrict__ lexp,
                                               int64_t *__restrict__ n_accept) {
    using O = RowOps<T, CHI>;
    extern __shared__ uint8_t sm_spins[];
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    const int grp = threadIdx.x / O::G;  // group in block
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const bool active = c0 < B;
    const int64_t c = active ? c0 : B - 1;
    uint8_t *s = sm_spins + (size_t)grp * a.N;
    for (int i = gl; i < a.N; i += O::G) s[i] = spins[c * a.N + i];
    __syncwarp();
    const T *A = (const T *)a.A;
    T *rst = rstack + (size_t)c * a.N * CHI;
    int32_t *rex = rexp + (size_t)c * a.N;
    double pm = state[c].mant;
    int64_t pe = state[c].exp2;
    int64_t acc_count = 0;
    const int span = (a.R - 1) * a.N;  // sites after the first one of a flip row
    for (int sw = 0; sw < n_sweeps; ++sw) {
        // right environments from the current spins (own chain only: active
        // groups write, inactive ones compute but never store)
        right_env_chain<T, CHI>(a, s, rst, rex, active, gl);
        __syncwarp();
        T l[O::NQ];
        O::load((const T *)a.bl, l, gl);
        int64_t El = 0;
        for (int j = 0; j < a.N; ++j) {
            const int i = __ldg(a.q + j);
            const int si = s[i];
            T u[O::NQ], keep[O::NQ];
            O::vecmat(site<T, CHI>(A, j, si ^ 1), l, u, gl);
            const int64_t Eu0 = El + O::renorm(u);
            O::vecmat(site<T, CHI>(A, j, si), l, keep, gl);
            const int64_t Ek = El + O::renorm(keep);
            T uf[O::NQ];
#pragma unroll
            for (int qq = 0; qq < O::NQ; ++qq) uf[qq] = u[qq];
            int64_t Eu = Eu0;
            int t = j + 1 == a.N ? 0 : j + 1;
            for (int k = j + 1; k <= j + span; ++k) {
                const int sp = s[__ldg(a.q + t)] ^ ((t == j) ? 1 : 0);
                O::vecmat(site<T, CHI>(A, k, sp), u, u, gl);
                Eu += O::renorm(u);
                if (++t == a.N) t = 0;
            }
            T r[O::NQ];
            O::load(rst + (size_t)j * CHI, r, gl);
            Eu += rex[j];
            double m = O::dot(u, r);
            normalize_scalar(m, Eu);
            const double ratio = ldexp(m / pm, (int)(Eu - pe));
            const double x = mcmc_uniform(seed, (uint64_t)(chain0 + c), (uint64_t)(sweep0 + sw),
                                          (uint64_t)j);
            const bool accept = x < ratio * ratio;
            if (accept) {
                pm = m;
                pe = Eu;
                ++acc_count;
#pragma unroll
                for (int qq = 0; qq < O::NQ; ++qq) l[qq] = uf[qq];
                El = Eu0;
            } else {
#pragma unroll
                for (int qq = 0; qq < O::NQ; ++qq) l[qq] = keep[qq];
                El = Ek;
            }
            __syncwarp();
            if (accept && gl == 0) s[i] = (uint8_t)(si ^ 1);
            __syncwarp();
            if (lstack && sw == n_sweeps - 1 && active) {
                O::store(lstack + ((size_t)c * a.N + j) * CHI, l, gl);
                if (gl == 0) lexp[(size_t)c * a.N + j] = (int32_t)El;
            }
        }
    }
    __syncwarp();
    if (active) {
        for (int i = gl; i < a.N; i += O::G) spins[c * a.N + i] = s[i];
        if (gl == 0) {
            state[c].mant = pm;
            state[c].exp2 = pe;
            if (n_accept) n_accept[c] += acc_count;
        }
    }
}

// ---------------------------------------------------------------------------
// General paths.  Right environments r_k = A_k ... A_{L-1} b_R for k >= kmin
// (kmin = 1 + the smallest last site of a spin), from the current spins, one
// group per chain: entry e holds r_{kmin+e}, entry L-kmin is b_R.
// ---------------------------------------------------------------------------
template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_right_env_gen(KArgs a, const uint8_t *__restrict__ spins,
                                                       int64_t B, T *__restrict__ rstack,
                                                       int32_t *__restrict__ rexp) {
    using O = RowOps<T, CHI>;
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const bool active = c0 < B;
    const int64_t c = active ? c0 : B - 1;
    const int nr = a.L - a.kmin + 1;
    const uint8_t *s = spins + c * a.N;
    T *rst = rstack + (size_t)c * nr * CHI;
    int32_t *rex = rexp + (size_t)c * nr;
    const T *AT = (const T *)a.AT;
    T r[O::NQ];
    O::load((const T *)a.br, r, gl);
    int32_t E = 0;
    if (active) {
        O::store(rst + (size_t)(nr - 1) * CHI, r, gl);
        if (gl == 0) rex[nr - 1] = 0;
    }
    for (int k = a.L - 1; k >= a.kmin; --k) {
        O::vecmat(site<T, CHI>(AT, k, __ldg(s + __ldg(a.p + k))), r, r, gl);
        E += O::renorm(r);
        if (active) {
            O::store(rst + (size_t)(k - a.kmin) * CHI, r, gl);
            if (gl == 0) rex[k - a.kmin] = E;
        }
    }
}

// Rows on a general path: group (c, j), j in [0, N].  j < N flips spin
// i = p[j] (first site j): l_{j-1} . A_j[s'] ... A_last[i][s'] . r_{last[i]+1};
// j = N: psi(s) = l_{N-1} . A_N ... A_{L-1} . b_R.  The groups of a warp share
// j, hence the loop length.
template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_rows_gen(KArgs a, const uint8_t *__restrict__ spins,
                                                  int64_t B, const T *__restrict__ lstack,
                                                  const int32_t *__restrict__ lexp,
                                                  const T *__restrict__ rstack,
                                                  const int32_t *__restrict__ rexp,
                                                  double *__restrict__ rows_mant,
                                                  int64_t *__restrict__ rows_exp) {
    using O = RowOps<T, CHI>;
    constexpr int RPW = Geo<CHI>::RPW;
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const int64_t n_cb = (B + RPW - 1) / RPW;
    const int64_t total = n_cb * (a.N + 1) * RPW;
    const int64_t gg = g0 < total ? g0 : total - 1;
    const int r_in = (int)(gg % RPW);
    const int j = (int)((gg / RPW) % (a.N + 1));
    const int64_t c0 = (gg / RPW / (a.N + 1)) * RPW + r_in;
    const bool active = g0 < total && c0 < B;
    const int64_t c = c0 < B ? c0 : B - 1;
    const int64_t g = c * (a.N + 1) + j;
    const uint8_t *s = spins + c * a.N;
    const T *A = (const T *)a.A;
    const int nr = a.L - a.kmin + 1;
    const int i = (j < a.N) ? __ldg(a.p + j) : -1;
    T u[O::NQ];
    int64_t E;
    if (j == 0) {
        O::load((const T *)a.bl, u, gl);
        E = 0;
    } else {
        O::load(lstack + ((size_t)c * a.N + (j - 1)) * CHI, u, gl);
        E = lexp[(size_t)c * a.N + (j - 1)];
    }
    const int end = (j < a.N) ? __ldg(a.last + i) : a.L - 1;
    for (int k = j; k <= end; ++k) {
        const int pk = __ldg(a.p + k);
        const int sp = __ldg(s + pk) ^ ((pk == i) ? 1 : 0);
        O::vecmat(site<T, CHI>(A, k, sp), u, u, gl);
        E += O::renorm(u);
    }
    const int e = end + 1 - a.kmin;  // r_{end+1}; b_R for j = N
    T r[O::NQ];
    O::load(rstack + ((size_t)c * nr + e) * CHI, r, gl);
    E += rexp[(size_t)c * nr + e];
    double m = O::dot(u, r);
    normalize_scalar(m, E);
    if (active && gl == 0) {
        rows_mant[g] = m;
        rows_exp[g] = E;
    }
}

// Metropolis sweeps on a general path, one group per chain.  Proposal j flips
// spin i = p[j]: the row runs from l_{j-1} (kept as in k_sweep) through
// last[i]; the right part r_{last[i]+1} is rebuilt from b_R with the current
// spins (sites after last[i] may carry spins flipped earlier in the sweep), as
// the oracle's from-scratch flip amplitude does.
template <typename T, int CHI>
__global__ void __launch_bounds__(256) k_sweep_gen(KArgs a, uint8_t *__restrict__ spins,
                                                   rtt_chain_state *__restrict__ state, int64_t B,
                                                   int64_t chain0, int64_t sweep0, int n_sweeps,
                                                   uint64_t seed, int64_t *__restrict__ n_accept) {
    using O = RowOps<T, CHI>;
    extern __shared__ uint8_t sm_spins[];
    const int lane = threadIdx.x & 31, gl = lane % O::G;
    const int grp = threadIdx.x / O::G;
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / O::G;
    const bool active = c0 < B;
    const int64_t c = active ? c0 : B - 1;
    uint8_t *s = sm_spins + (size_t)grp * a.N;
    for (int i = gl; i < a.N; i += O::G) s[i] = spins[c * a.N + i];
    __syncwarp();
    const T *A = (const T *)a.A;
    const T *AT = (const T *)a.AT;
    double pm = state[c].mant;
    int64_t pe = state[c].exp2;
    int64_t acc_count = 0;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        T l[O::NQ];
        O::load((const T *)a.bl, l, gl);
        int64_t El = 0;
        for (int j = 0; j < a.N; ++j) {
            const int i = __ldg(a.p + j);
            const int si = s[i];
            const int last = __ldg(a.last + i);
            T u[O::NQ], keep[O::NQ];
            O::vecmat(site<T, CHI>(A, j, si ^ 1), l, u, gl);
            const int64_t Eu0 = El + O::renorm(u);
            O::vecmat(site<T, CHI>(A, j, si), l, keep, gl);
            const int64_t Ek = El + O::renorm(keep);
            T uf[O::NQ];
#pragma unroll
            for (int qq = 0; qq < O::NQ; ++qq) uf[qq] = u[qq];
            int64_t Eu = Eu0;
            for (int k = j + 1; k <= last; ++k) {
                const int pk = __ldg(a.p + k);
                const int sp = s[pk] ^ ((pk == i) ? 1 : 0);
                O::vecmat(site<T, CHI>(A, k, sp), u, u, gl);
                Eu += O::renorm(u);
            }
            T r[O::NQ];
            O::load((const T *)a.br, r, gl);
            for (int k = a.L - 1; k > last; --k) {
                O::vecmat(site<T, CHI>(AT, k, s[__ldg(a.p + k)]), r, r, gl);
                Eu += O::renorm(r);
            }
            double m = O::dot(u, r);
            normalize_scalar(m, Eu);
            const double ratio = ldexp(m / pm, (int)(Eu - pe));
            const double x = mcmc_uniform(seed, (uint64_t)(chain0 + c), (uint64_t)(sweep0 + sw),
                                          (uint64_t)j);
            const bool accept = x < ratio * ratio;
            if (accept) {
                pm = m;
                pe = Eu;
                ++acc_count;
#pragma unroll
                for (int qq = 0; qq < O::NQ; ++qq) l[qq] = uf[qq];
                El = Eu0;
            } else {
#pragma unroll
                for (int qq = 0; qq < O::NQ; ++qq) l[qq] = keep[qq];
                El = Ek;
            }
            __syncwarp();
            if (accept && gl == 0) s[i] = (uint8_t)(si ^ 1);
            __syncwarp();
        }
    }
    __syncwarp();
    if (active) {
        for (int i = gl; i < a.N; i += O::G) spins[c * a.N + i] = s[i];
        if (gl == 0) {
            state[c].mant = pm;
            state[c].exp2 = pe;
            if (n_accept) n_accept[c] += acc_count;
        }
    }
}

// ---------------------------------------------------------------------------
// host-side dispatch over CHI
// ---------------------------------------------------------------------------
template <typename T>
struct SimtLaunch {
    template <int CHI>
    static int64_t blocks_for(int64_t groups) {
        const int64_t per_block = 256 / Geo<CHI>::G;
        return (groups + per_block - 1) / per_block;
    }

    template <int CHI>
    static cudaError_t run(int which, const SimtArgs &sa, const void *p0, void *p1, void *p2,
                           void *p3, void *p4, void *p5, void *p6, int64_t B, int64_t i0,
                           int64_t i1, int32_t i2, uint64_t u0, cudaStream_t st) {
        KArgs a{sa.A, sa.AT, sa.bl, sa.br, sa.q, sa.N, sa.L, sa.R, sa.p, sa.last, sa.kmin};
        switch (which) {
            case 0:
                k_left_env<T, CHI><<<(unsigned)blocks_for<CHI>(B), 256, 0, st>>>(
                    a, (const uint8_t *)p0, B, (T *)p1, (int32_t *)p2);
                break;
            case 1:
                if (sa.p)
                    k_right_env_gen<T, CHI><<<(unsigned)blocks_for<CHI>(B), 256, 0, st>>>(
                        a, (const uint8_t *)p0, B, (T *)p1, (int32_t *)p2);
                else
                    k_right_env<T, CHI><<<(unsigned)blocks_for<CHI>(B), 256, 0, st>>>(
                        a, (const uint8_t *)p0, B, (T *)p1, (int32_t *)p2);
                break;
            case 2:
                if (sa.p) {
                k_rows_gen<T, CHI><<<(unsigned)blocks_for<CHI>(
                                     (B + Geo<CHI>::RPW - 1) / Geo<CHI>::RPW * (sa.N + 1) *
                                     Geo<CHI>::RPW),
                                 256, 0, st>>>(
                    a, (const uint8_t *)p0, B, (const T *)p1, (const int32_t *)p2,
                    (const T *)p3, (const int32_t *)p4, (double *)p5, (int64_t *)p6);
                } else {
                k_rows<T, CHI><<<(unsigned)blocks_for<CHI>(
                                     (B + Geo<CHI>::RPW - 1) / Geo<CHI>::RPW * (sa.N + 1) *
                                     Geo<CHI>::RPW),
                                 256, 0, st>>>(
                    a, (const uint8_t *)p0, B, (const T *)p1, (const int32_t *)p2,
                    (const T *)p3, (const int32_t *)p4, (double *)p5, (int64_t *)p6);
                }
                break;
            case 3:
                k_chain_init<T, CHI><<<(unsigned)blocks_for<CHI>(B), 256, 0, st>>>(
                    a, (const uint8_t *)p0, B, (double *)p1, (int8_t *)p2, (rtt_chain_state *)p3);
                break;
            case 4: {
                const size_t smem = (size_t)(256 / Geo<CHI>::G) * sa.N;
                if (smem > 48 * 1024) {
                    cudaError_t e = cudaFuncSetAttribute(k_sweep<T, CHI>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)smem);
                    if (e != cudaSuccess) return e;
                }
                if (sa.p) {
                    if (smem > 48 * 1024) {
                        cudaError_t e = cudaFuncSetAttribute(
                            k_sweep_gen<T, CHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                        if (e != cudaSuccess) return e;
                    }
                    k_sweep_gen<T, CHI><<<(unsigned)blocks_for<CHI>(B), 256, smem, st>>>(
                        a, (uint8_t *)p0, (rtt_chain_state *)p1, B, i0, i1, i2, u0, (int64_t *)p6);
                } else {
                    k_sweep<T, CHI><<<(unsigned)blocks_for<CHI>(B), 256, smem, st>>>(
                        a, (uint8_t *)p0, (rtt_chain_state *)p1, B, i0, i1, i2, u0, (T *)p2,
                        (int32_t *)p3, (T *)p4, (int32_t *)p5, (int64_t *)p6);
                }
                break;
            }
            default:
                return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }

    static cudaError_t dispatch(int which, const SimtArgs &sa, const void *p0, void *p1, void *p2,
                                void *p3, void *p4, void *p5, void *p6, int64_t B, int64_t i0 = 0,
                                int64_t i1 = 0, int32_t i2 = 0, uint64_t u0 = 0,
                                cudaStream_t st = 0) {
        switch (sa.chip) {
            case 1: return run<1>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 2: return run<2>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 4: return run<4>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 8: return run<8>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 16: return run<16>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 32: return run<32>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 64: return run<64>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 128: return run<128>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            case 256: return run<256>(which, sa, p0, p1, p2, p3, p4, p5, p6, B, i0, i1, i2, u0, st);
            default: return cudaErrorInvalidValue;
        }
    }
};

}  // namespace rttd

#define RTT_DEFINE_SIMT(T, SUFFIX)                                                                 \
    cudaError_t simt_left_env_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,         \
                                       void *lstack, int32_t *lexp, cudaStream_t st) {             \
        return rttd::SimtLaunch<T>::dispatch(0, a, spins, lstack, lexp, nullptr, nullptr, nullptr, \
                                             nullptr, B, 0, 0, 0, 0, st);                          \
    }                                                                                              \
    cudaError_t simt_right_env_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,        \
                                        void *rstack, int32_t *rexp, cudaStream_t st) {            \
        return rttd::SimtLaunch<T>::dispatch(1, a, spins, rstack, rexp, nullptr, nullptr, nullptr, \
                                             nullptr, B, 0, 0, 0, 0, st);                          \
    }                                                                                              \
    cudaError_t simt_rows_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,             \
                                   const void *lstack, const int32_t *lexp, const void *rstack,    \
                                   const int32_t *rexp, double *rows_mant, int64_t *rows_exp,      \
                                   cudaStream_t st) {                                              \
        return rttd::SimtLaunch<T>::dispatch(2, a, spins, (void *)lstack, (void *)lexp,            \
                                             (void *)rstack, (void *)rexp, rows_mant, rows_exp, B, \
                                             0, 0, 0, 0, st);                                      \
    }                                                                                              \
    cudaError_t simt_chain_init_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,       \
                                         double *log_abs, int8_t *sign, rtt_chain_state *state,    \
                                         cudaStream_t st) {                                        \
        return rttd::SimtLaunch<T>::dispatch(3, a, spins, log_abs, sign, state, nullptr, nullptr,  \
                                             nullptr, B, 0, 0, 0, 0, st);                          \
    }                                                                                              \
    cudaError_t simt_sweep_##SUFFIX(const SimtArgs &a, uint8_t *spins, rtt_chain_state *state,     \
                                    int64_t B, int64_t chain0, int64_t sweep0, int32_t n_sweeps,   \
                                    uint64_t seed, void *rstack, int32_t *rexp, void *lstack,      \
                                    int32_t *lexp, int64_t *n_accept, cudaStream_t st) {           \
        return rttd::SimtLaunch<T>::dispatch(4, a, spins, state, rstack, rexp, lstack, lexp,       \
                                             n_accept, B, chain0, sweep0, n_sweeps, seed, st);     \
    }
