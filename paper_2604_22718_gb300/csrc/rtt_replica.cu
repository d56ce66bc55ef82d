// rtt_replica.cu -- replica-space optimization (Sec. 3.1): lifting of Pauli
// terms through the Kronecker part C (Sec. 2.2.3), and (1 - tau H-bar) on
// tensor trains as a tree of two-term sums, each rounded back to rank chi.
//
// Device work is one kernel, k_tt_round: one warp rounds one two-term sum.
//   sweep 1 (left to right): the block-diagonal sum core, with the terms'
//     Pauli strings applied while it is loaded, is multiplied by the R factor
//     carried from the previous site and factored by Householder QR; Q goes to
//     global scratch (it is read back once by sweep 2, mostly from L2), R is
//     carried on;
//   sweep 2 (right to left): each core, with the factor U S carried from the
//     site to its right, is unfolded (rows: left bond; columns: physical index
//     and right bond) and decomposed by one-sided Jacobi (Hestenes): the
//     columns are rotated pairwise until orthogonal, so the rotated columns
//     are U S and the accumulated rotations V.  The chi largest singular
//     values are kept: rows of V^T become the output core, U S is carried on.
// Lanes own matrix columns (at most 2 chi <= 32 of them) in registers: a
// reflector or a rotation is one unrolled loop per lane, the reflectors pass
// through shared memory and a Jacobi partner's column comes by shuffle.  The
// arithmetic is FP64 or FP32 (the cores stay FP64 in memory); the TT's scale
// travels as an integer power-of-two exponent, so FP32 cannot overflow on long
// trains.  A rounding is a chain of 2 L small dependent factorizations, bound
// by latency rather than arithmetic throughput.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rtt_internal.cuh"

namespace {

constexpr int kMaxChi = 16;

struct TTItem {
    const double *tt;     // padded cores [L][2][chi][chi]
    const uint8_t *ops;   // string codes [L] or null (identity)
    double coef;          // multiplies the first core
    int chi;              // this TT's padded rank (its cores' layout)
};
struct TTPair {
    TTItem a, b;
    double *out;          // padded cores [L][2][chi_out][chi_out]
    int chi_out;          // rank the sum is rounded to
};

rtt_status rp_fail(rtt_status s, const std::string &msg) {
    rtt_set_error(msg);
    return s;
}

// Per-warp shared memory, T = arithmetic type, CM = compile-time bound on chi:
// the Householder vectors of the current site and the R factor carried to the
// next one.  Everything else lives in registers, one matrix column per lane.
template <typename T, int CM>
struct WarpSmem {
    static constexpr int D2 = 2 * CM, MR = 4 * CM;
    T v[D2][MR];        // sweep 1: Householder vectors (zero above their pivot)
    T beta[D2];
    T r[D2][D2];        // R factor carried to the next site (row-major)
};

template <typename T> struct Arith;
// eps: unit roundoff x 2, times the column length the Jacobi threshold; big: the
// largest zeta whose square is finite; tiny: a column whose squared norm is
// below it counts as zero in the QR (v^T v >= 2 |x|^2, so 2 / v^T v stays
// finite; at the O(1) scale of these matrices such a column is far below the
// type's resolution).
template <> struct Arith<double> {
    static constexpr double eps = 2.220446049250313e-16;
    static constexpr double big = 1e150;
    static constexpr double tiny = 1e-290;
};
template <> struct Arith<float> {
    static constexpr float eps = 1.1920929e-7f;
    static constexpr float big = 1e18f;
    static constexpr float tiny = 1e-30f;
};

// floor(log2 x) of a finite x > 0 from its exponent field, clamped so that
// pow2<T>(-e) stays a normal number; pow2<T>(e) = 2^e exactly.
__device__ __forceinline__ int exp2_of(float x) {
    const int e = (int)((__float_as_uint(x) >> 23) & 0xffu) - 127;
    return max(-125, min(125, e));
}
__device__ __forceinline__ int exp2_of(double x) {
    const int e = (int)((unsigned long long)(__double_as_longlong(x) >> 52) & 0x7ffull) - 1023;
    return max(-1021, min(1021, e));
}
template <typename T> __device__ __forceinline__ T pow2(int e);
template <> __device__ __forceinline__ float pow2<float>(int e) {
    return __uint_as_float((unsigned)(127 + e) << 23);
}
template <> __device__ __forceinline__ double pow2<double>(int e) {
    return __longlong_as_double((long long)(1023 + e) << 52);
}

// Element (b, s, c) of the sum core at site k: block diagonal in the middle,
// [a | b] at the first site, [a ; b] stacked at the last; strings applied.
// The first cores are scaled by s0 (an exact power of two) in FP64 before the
// conversion to T, so that a TT whose norm sits in its first core cannot
// overflow the arithmetic type.
template <typename T>
__device__ __forceinline__ T item_core(const TTItem &it, int L, int k, int s, int b, int c,
                                       double s0) {
    const int chi = it.chi;
    int so = s;
    double sg = 1.0;
    if (it.ops) {
        const uint8_t op = it.ops[k];
        if (op == 1) so = 1 - s;
        else if (op == 2 && s == 1) sg = -1.0;
    }
    if (k == 0) sg *= it.coef * s0;
    return (T)(sg * it.tt[(((size_t)k * 2 + so) * chi + b) * chi + c]);
}

template <typename T>
__device__ __forceinline__ T sum_core(const TTItem &A, const TTItem &B, int L, int k, int s, int b,
                                      int c, double s0) {
    const int dA = A.chi;                 // A's block comes first
    if (k == 0) {                         // left rank 1
        return c < dA ? item_core<T>(A, L, k, s, 0, c, s0) : item_core<T>(B, L, k, s, 0, c - dA, s0);
    }
    if (k == L - 1) {                     // right rank 1
        return b < dA ? item_core<T>(A, L, k, s, b, 0, s0) : item_core<T>(B, L, k, s, b - dA, 0, s0);
    }
    if (b < dA && c < dA) return item_core<T>(A, L, k, s, b, c, s0);
    if (b >= dA && c >= dA) return item_core<T>(B, L, k, s, b - dA, c - dA, s0);
    return T(0);
}

template <typename T, int CM>
__global__ void __launch_bounds__(128) k_tt_round(const TTPair *__restrict__ pairs, int npairs,
                                                  int L, T *__restrict__ scratch,
                                                  int normalize, double *__restrict__ log_norm) {
    constexpr int D2M = 2 * CM, MR = 4 * CM;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    if (w >= npairs) return;
    WarpSmem<T, CM> &S = reinterpret_cast<WarpSmem<T, CM> *>(smem_raw)[wib];
    const TTPair P = pairs[w];
    const int D2 = P.a.chi + P.b.chi;            // bond of the sum
    const int chi = P.chi_out;                   // rank (and layout) of the result
    const size_t qstride = (size_t)2 * D2M * D2M;            // one site's Q, [row (a,s)][col]
    T *Q = scratch + (size_t)w * L * qstride;

    // Power-of-two bookkeeping: the TT's scale is carried as an integer
    // exponent E (a TT of ones on 144 sites has norm 2^72, whose square
    // exceeds the FP32 range).  First the first cores, scaled on load ...
    int E = 0;
    double s0 = 1.0;
    {
        double mx = 0.0;
        for (int e = lane; e < 2 * P.a.chi; e += 32) {
            const int s = e / P.a.chi, c = e % P.a.chi;
            mx = fmax(mx, fabs(P.a.coef * P.a.tt[(s * P.a.chi + 0) * P.a.chi + c]));
        }
        for (int e = lane; e < 2 * P.b.chi; e += 32) {
            const int s = e / P.b.chi, c = e % P.b.chi;
            mx = fmax(mx, fabs(P.b.coef * P.b.tt[(s * P.b.chi + 0) * P.b.chi + c]));
        }
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, off));
        if (mx > 0.0 && isfinite(mx)) {
            E = exp2_of(mx);
            s0 = pow2<double>(-E);
        }
    }

    // ---------------- sweep 1: left to right, Householder QR -----------------
    // Lane c holds column c of M = R x_1 G_k in col[], rows (a, s) -> a * 2 + s.
    // R starts as the 1 x 1 identity (left rank 1 at the first site).
    if (lane == 0) S.r[0][0] = T(1);
    __syncwarp();
    int rl = 1;                                  // rows of R = left rank of M
    T col[MR];
    for (int k = 0; k < L; ++k) {
        const int dl = (k == 0) ? 1 : D2;        // left bond of the sum core
        const int dr = (k == L - 1) ? 1 : D2;    // right bond
        const int mr = 2 * rl;
#pragma unroll
        for (int i = 0; i < MR; ++i) col[i] = T(0);
        if (lane < dr) {
            for (int b = 0; b < dl; ++b) {
                const T g0 = sum_core<T>(P.a, P.b, L, k, 0, b, lane, s0);
                const T g1 = sum_core<T>(P.a, P.b, L, k, 1, b, lane, s0);
#pragma unroll
                for (int a = 0; a < D2M; ++a)
                    if (a < rl) {
                        const T rab = S.r[a][b];
                        col[2 * a] = fma(rab, g0, col[2 * a]);
                        col[2 * a + 1] = fma(rab, g1, col[2 * a + 1]);
                    }
            }
        }
        // ... then M at every site: its largest entry brought into [1, 2)
        {
            T mx = T(0);
#pragma unroll
            for (int i = 0; i < MR; ++i)
                if (i < mr) mx = fmax(mx, fabs(col[i]));
            for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, off));
            if (mx > T(0) && isfinite(mx)) {
                const int e = exp2_of(mx);
                if (e != 0) {
                    const T f = pow2<T>(-e);
#pragma unroll
                    for (int i = 0; i < MR; ++i) col[i] *= f;
                    E += e;
                }
            }
        }
        __syncwarp();                            // S.r is rewritten below
        T *Qk = Q + (size_t)k * qstride;
        if (k == L - 1) {                        // the last core keeps R absorbed
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < MR; ++i)
                    if (i < mr) Qk[(size_t)i * D2M] = col[i];
            }
            __syncwarp();                        // lane 1 reads this core in sweep 2
            break;
        }
        const int m = min(mr, dr);
        for (int j = 0; j < m; ++j) {
            if (lane == j) {
                T n2 = T(0), x0 = T(0);
#pragma unroll
                for (int i = 0; i < MR; ++i) {
                    if (i >= j && i < mr) n2 = fma(col[i], col[i], n2);
                    if (i == j) x0 = col[i];
                }
                T beta = T(0), alpha = T(0), v0 = T(0);
                const bool live = n2 > Arith<T>::tiny;
                if (live) {
                    alpha = x0 >= T(0) ? -sqrt(n2) : sqrt(n2);
                    v0 = x0 - alpha;
                    const T vtv = n2 - x0 * x0 + v0 * v0;
                    beta = vtv > T(0) ? T(2) / vtv : T(0);
                }
#pragma unroll
                for (int i = 0; i < MR; ++i) {
                    T vi = T(0);
                    if (live && i > j && i < mr) vi = col[i];
                    if (live && i == j) vi = v0;
                    S.v[j][i] = vi;
                    if (i == j) col[i] = live ? alpha : x0;
                    else if (i > j && live) col[i] = T(0);
                }
                S.beta[j] = beta;
            }
            __syncwarp();
            if (lane > j && lane < dr) {
                const T beta = S.beta[j];
                T d = T(0);
#pragma unroll
                for (int i = 0; i < MR; ++i)
                    if (i < mr) d = fma(S.v[j][i], col[i], d);
                d *= beta;
#pragma unroll
                for (int i = 0; i < MR; ++i)
                    if (i < mr) col[i] = fma(-d, S.v[j][i], col[i]);
            }
        }
        // R (m x dr, upper trapezoidal) for the next site: rows j < m of the columns
        if (lane < dr) {
#pragma unroll
            for (int j = 0; j < D2M; ++j)
                if (j < m) S.r[j][lane] = col[j];
        }
        // Q = H_0 ... H_{m-1} I[:, :m], lane c < m builds column c
        if (lane < m) {
#pragma unroll
            for (int i = 0; i < MR; ++i) col[i] = (i == lane) ? T(1) : T(0);
            for (int j = m - 1; j >= 0; --j) {
                const T beta = S.beta[j];
                T d = T(0);
#pragma unroll
                for (int i = 0; i < MR; ++i)
                    if (i < mr) d = fma(S.v[j][i], col[i], d);
                d *= beta;
#pragma unroll
                for (int i = 0; i < MR; ++i)
                    if (i < mr) col[i] = fma(-d, S.v[j][i], col[i]);
            }
#pragma unroll
            for (int i = 0; i < MR; ++i)
                if (i < mr) Qk[(size_t)i * D2M + lane] = col[i];
        }
        __syncwarp();                            // S.v, S.beta, S.r complete
        rl = m;
    }

    // ---------------- sweep 2: right to left, truncated SVD ------------------
    // Lane j holds column j of the unfolding N (rows: left bond a < r0; columns
    // (s, c) -> s * r1 + c) in x[] and column j of the accumulated rotation V
    // in vc[]; the partner's columns come by shuffle.
    auto rank_left = [&](int k) { return k >= 5 ? D2 : min(1 << k, D2); };
    double *out = P.out;
    int r1 = 1;
    T x[D2M], vc[D2M];
    {
        const int r0 = rank_left(L - 1);
        const T *Qk = Q + (size_t)(L - 1) * qstride;
#pragma unroll
        for (int a = 0; a < D2M; ++a)
            x[a] = (lane < 2 && a < r0) ? Qk[(size_t)(a * 2 + lane) * D2M] : T(0);
    }
    for (int k = L - 1; k >= 1; --k) {
        const int r0 = rank_left(k);
        const int n2 = 2 * r1;
#pragma unroll
        for (int i = 0; i < D2M; ++i) vc[i] = (i == lane) ? T(1) : T(0);
        // Hestenes sweeps with a round-robin tournament (n2 even): player 0
        // fixed, players 1..n2-1 rotate by one position per round
        for (int sweep = 0; sweep < 30; ++sweep) {
            int rotated = 0;
            for (int rnd = 0; rnd < n2 - 1; ++rnd) {
                int partner = lane;
                if (lane < n2) {
                    int pos = 0;
                    if (lane > 0) {
                        pos = lane - 1 - rnd;
                        if (pos < 0) pos += n2 - 1;
                        pos += 1;
                    }
                    const int ppos = n2 - 1 - pos;
                    if (ppos == 0) {
                        partner = 0;
                    } else {
                        int q = ppos - 1 + rnd;
                        if (q >= n2 - 1) q -= n2 - 1;
                        partner = q + 1;
                    }
                }
                T px[D2M], pv[D2M];
#pragma unroll
                for (int i = 0; i < D2M; ++i) {
                    px[i] = __shfl_sync(FULL, x[i], partner);
                    pv[i] = __shfl_sync(FULL, vc[i], partner);
                }
                if (lane < n2) {
                    const bool am_lo = lane < partner;
                    T a = T(0), b = T(0), g = T(0);
#pragma unroll
                    for (int i = 0; i < D2M; ++i)
                        if (i < r0) {
                            const T xl = am_lo ? x[i] : px[i], xh = am_lo ? px[i] : x[i];
                            a = fma(xl, xl, a);
                            b = fma(xh, xh, b);
                            g = fma(xl, xh, g);
                        }
                    // rotate while the columns are not orthogonal to the working
                    // precision: the computed g carries about r0 roundings of its own
                    T c = T(1), sn = T(0);
                    const T tol = Arith<T>::eps * T(r0);
                    if (g != T(0) && g * g > tol * tol * a * b) {
                        const T zeta = (b - a) / (T(2) * g);
                        // smaller root of t^2 + 2 zeta t - 1 = 0; 1/(2 zeta) once zeta^2 would overflow
                        const T t = fabs(zeta) > Arith<T>::big
                                        ? T(0.5) / zeta
                                        : (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                        c = T(1) / sqrt(T(1) + t * t);
                        sn = c * t;
                        rotated = 1;
                    }
                    // lo' = c lo - s hi, hi' = s lo + c hi
#pragma unroll
                    for (int i = 0; i < D2M; ++i) {
                        const T xl = am_lo ? x[i] : px[i], xh = am_lo ? px[i] : x[i];
                        x[i] = am_lo ? (c * xl - sn * xh) : (sn * xl + c * xh);
                        const T vl = am_lo ? vc[i] : pv[i], vh = am_lo ? pv[i] : vc[i];
                        vc[i] = am_lo ? (c * vl - sn * vh) : (sn * vl + c * vh);
                    }
                }
            }
            if (!__any_sync(FULL, rotated)) break;
        }
        // singular values and ranks (largest first, ties by index)
        T s2 = T(0);
#pragma unroll
        for (int i = 0; i < D2M; ++i)
            if (i < r0) s2 = fma(x[i], x[i], s2);
        const T sig = lane < n2 ? sqrt(s2) : T(-1);
        int rank = 0;
        for (int j = 0; j < n2; ++j) {
            const T sj = __shfl_sync(FULL, sig, j);
            rank += (sj > sig) || (sj == sig && j < lane);
        }
        const int t = min(chi, min(r0, n2));
        // output core k: row i < t is the V column of the lane ranked i; rows t..chi-1 zero
        double *ok = out + (size_t)k * 2 * chi * chi;
        if (lane < n2 && rank < t) {
#pragma unroll
            for (int e = 0; e < D2M; ++e)
                if (e < n2) {
                    const int s = e >= r1 ? 1 : 0, c = e - s * r1;
                    ok[(s * chi + rank) * chi + c] = (double)vc[e];
                }
            for (int s = 0; s < 2; ++s)
                for (int c = r1; c < chi; ++c) ok[(s * chi + rank) * chi + c] = 0.0;
        }
        if (lane >= t && lane < chi)
            for (int s = 0; s < 2; ++s)
                for (int c = 0; c < chi; ++c) ok[(s * chi + lane) * chi + c] = 0.0;
        // next N = Q_{k-1} (r0' x 2 x r0) x_3 (U S)(r0 x t), column (s, i) -> s * t + i,
        // U S column i = rotated column of the lane ranked i
        const int nn = 2 * t;
        const int my_i = lane < nn ? (lane >= t ? lane - t : lane) : 0;
        const int my_s = lane < nn && lane >= t ? 1 : 0;
        int my_sel = 0;
        for (int i = 0; i < t; ++i) {
            const unsigned m = __ballot_sync(FULL, lane < n2 && rank == i);
            if (i == my_i) my_sel = __ffs(m) - 1;
        }
        T wcol[D2M];
#pragma unroll
        for (int b = 0; b < D2M; ++b) wcol[b] = __shfl_sync(FULL, x[b], my_sel);
        const int rp = rank_left(k - 1);
        const T *Qp = Q + (size_t)(k - 1) * qstride;
#pragma unroll
        for (int a = 0; a < D2M; ++a) {
            T acc = T(0);
            if (lane < nn && a < rp) {
#pragma unroll
                for (int b = 0; b < D2M; ++b)
                    if (b < r0) acc = fma(Qp[(size_t)(a * 2 + my_s) * D2M + b], wcol[b], acc);
            }
            x[a] = acc;
        }
        r1 = t;
    }
    // first core: 1 x 2 x r1 in x[0] of lanes < 2 r1, times 2^E; or scaled to
    // unit norm (the norm's log then takes E ln 2)
    double scale = pow2<double>(E);
    if (normalize) {
        T s2 = T(0);
        for (int j = 0; j < 2 * r1; ++j) {
            const T v = __shfl_sync(FULL, x[0], j);
            s2 = fma(v, v, s2);
        }
        const T nrm = sqrt(s2);
        scale = 1.0 / (double)nrm;
        if (lane == 0 && log_norm) log_norm[w] = log((double)nrm) + (double)E * 0.6931471805599453;
    }
    if (lane < 2 * r1) {
        const int s = lane >= r1 ? 1 : 0, c = lane - s * r1;
        out[(s * chi + 0) * chi + c] = (double)x[0] * scale;
    }
    // the rest of core 0 is zero: rows 1.., and columns r1.. of row 0
    for (int e = lane; e < 2 * chi * chi; e += 32) {
        const int i = (e / chi) % chi, c = e % chi;
        if (i != 0 || c >= r1) out[e] = 0.0;
    }
}

template <int CM>
constexpr int warps_per_cta() {
    return CM <= 8 ? 4 : 2;
}

// chi (below): the largest rank among the launch's TTs, which picks the
// compile-time bound CM (every sum's bond is at most 2 CM)
template <typename T, int CM>
cudaError_t launch_round(const TTPair *pairs, int npairs, int L, int chi, void *scratch,
                         int normalize, double *log_norm, cudaStream_t st) {
    (void)chi;
    constexpr int wpc = warps_per_cta<CM>();
    const size_t smem = sizeof(WarpSmem<T, CM>) * wpc;
    // per device and cheap: set on every launch
    cudaError_t e = cudaFuncSetAttribute(k_tt_round<T, CM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (npairs + wpc - 1) / wpc;
    k_tt_round<T, CM><<<blocks, 32 * wpc, smem, st>>>(pairs, npairs, L, (T *)scratch, normalize,
                                                      log_norm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_round_t(const TTPair *pairs, int npairs, int L, int chi, void *scratch,
                           int normalize, double *log_norm, cudaStream_t st) {
    if (chi <= 2) return launch_round<T, 2>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
    if (chi <= 4) return launch_round<T, 4>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
    if (chi <= 8) return launch_round<T, 8>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
    return launch_round<T, 16>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
}

cudaError_t launch_round_any(const TTPair *pairs, int npairs, int L, int chi, int precision,
                             void *scratch, int normalize, double *log_norm, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    if (precision == RTT_FP32)
        return launch_round_t<float>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
    return launch_round_t<double>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
}

}  // namespace

// ----------------------------------------------------------------------------
// Plan
// ----------------------------------------------------------------------------
struct rtt_tt_plan_s {
    int device = 0, L = 0, chi = 0, K = 0, precision = RTT_FP64;
    int chi_tree = 0;             // rank the tree's pairwise sums are rounded to
    int cm = 0;                   // the largest rank of the plan's TTs, max(chi, chi_tree)
    std::vector<double> eta;
    uint8_t *d_ops = nullptr;     // [K][L]
    double *d_nodes = nullptr;    // [K-1][L][2][chi_tree][chi_tree] tree node TTs
    double *d_next = nullptr;     // [L][2][chi][chi]
    void *d_scratch = nullptr;    // [max pairs][L][2 (2chi)^2] of the arithmetic type (padded
                                  // to the kernel's bound on chi)
    TTPair *d_pairs = nullptr;    // the tree's pairs, level by level, then the final pair
    std::vector<int> level_off;   // pairs of level l: [level_off[l], level_off[l+1])
    int max_pairs = 1;
    size_t qsite = 0;             // elements of one site's Q in the scratch
    const double *pairs_phi = nullptr;  // phi and tau the device pairs were built for
    double pairs_tau = 0.0;
    bool pairs_valid = false;
};

namespace {

size_t q_site_doubles(int chi) {
    const int cm = chi <= 2 ? 2 : (chi <= 4 ? 4 : (chi <= 8 ? 8 : 16));
    return (size_t)2 * (2 * cm) * (2 * cm);
}

// Pairs of the tree over `items` (two by two, an odd last item passes up),
// level by level, node outputs in the plan's node buffers in creation order;
// appends to `pairs`, sets the plan's level offsets and returns the root.
TTItem build_tree(rtt_tt_plan_s *p, std::vector<TTItem> items, std::vector<TTPair> &pairs) {
    const size_t tt = (size_t)p->L * 2 * p->chi_tree * p->chi_tree;
    pairs.clear();
    p->level_off.assign(1, 0);
    int node = 0;
    while (items.size() > 1) {
        std::vector<TTItem> nxt;
        for (size_t i = 0; i + 1 < items.size(); i += 2) {
            double *o = p->d_nodes + (size_t)node++ * tt;
            pairs.push_back(TTPair{items[i], items[i + 1], o, p->chi_tree});
            nxt.push_back(TTItem{o, nullptr, 1.0, p->chi_tree});
        }
        if (items.size() % 2) nxt.push_back(items.back());
        items.swap(nxt);
        p->level_off.push_back((int)pairs.size());
    }
    return items[0];
}

std::vector<TTItem> term_items(rtt_tt_plan_s *p, const double *phi, int chi_phi) {
    std::vector<TTItem> items(p->K);
    for (int k = 0; k < p->K; ++k) items[k] = TTItem{phi, p->d_ops + (size_t)k * p->L, p->eta[k], chi_phi};
    return items;
}

// (1 - tau H-bar): the tree's root S, then phi - tau S into the plan's next buffer.
void build_pairs(rtt_tt_plan_s *p, const double *phi, double tau, std::vector<TTPair> &pairs) {
    TTItem s = build_tree(p, term_items(p, phi, p->chi), pairs);
    s.coef *= -tau;
    pairs.push_back(TTPair{TTItem{phi, nullptr, 1.0, p->chi}, s, p->d_next, p->chi});
}

// Upload a pair table (pageable source: staged before the call returns, copied
// in stream order after earlier work that read the old table) and run it:
// every tree level, then the final pair, which is scaled to unit norm.
cudaError_t run_pairs(rtt_tt_plan_s *p, const std::vector<TTPair> &pairs, double *log_norm,
                      cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(p->d_pairs, pairs.data(), pairs.size() * sizeof(TTPair),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int nlev = (int)p->level_off.size() - 1;
    for (int l = 0; l < nlev; ++l) {
        const int n = p->level_off[l + 1] - p->level_off[l];
        if ((e = launch_round_any(p->d_pairs + p->level_off[l], n, p->L, p->cm, p->precision, p->d_scratch, 0,
                                  nullptr, st)) != cudaSuccess)
            return e;
    }
    return launch_round_any(p->d_pairs + p->level_off.back(), 1, p->L, p->cm, p->precision, p->d_scratch, 1,
                            log_norm, st);
}

}  // namespace

extern "C" {

rtt_status rtt_replica_lift(int32_t n_spins, int32_t length, const int32_t *path, int32_t n_terms,
                            const double *coef, const int32_t *block, const int32_t *offsets,
                            const int32_t *spins, const uint8_t *ops, uint8_t *ops_out,
                            double *eta_out) {
    if (n_spins < 1 || length < 1 || n_terms < 0 || !path || (n_terms > 0 && (!coef || !block ||
        !offsets || !ops_out || !eta_out)))
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: bad sizes or null pointer");
    if (length % n_spins)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: length is not a multiple of n_spins");
    const int nb = length / n_spins;
    // R[j][c] = site of spin j in block c
    std::vector<int> R((size_t)n_spins * nb, -1);
    for (int c = 0; c < nb; ++c)
        for (int pos = 0; pos < n_spins; ++pos) {
            const int j = path[c * n_spins + pos];
            if (j < 0 || j >= n_spins || R[(size_t)j * nb + c] >= 0)
                return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: block " + std::to_string(c) +
                                                        " of the path is not a permutation of the spins");
            R[(size_t)j * nb + c] = c * n_spins + pos;
        }
    if (n_terms > 0 && offsets[0] != 0)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: offsets[0] must be 0");
    std::vector<char> seen(n_spins, 0);
    for (int k = 0; k < n_terms; ++k) {
        const int f0 = offsets[k], f1 = offsets[k + 1];
        if (f1 < f0 || (f1 > f0 && (!spins || !ops)))
            return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: offsets must not decrease");
        if (block[k] < 0 || block[k] >= nb)
            return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: block out of range in term " +
                                                    std::to_string(k));
        uint8_t *row = ops_out + (size_t)k * length;
        std::fill(row, row + length, (uint8_t)0);
        for (int f = f0; f < f1; ++f) {
            const int j = spins[f];
            if (j < 0 || j >= n_spins)
                return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: spin out of range");
            if (seen[j]) {
                for (int g = f0; g < f; ++g) seen[spins[g]] = 0;
                return rp_fail(RTT_ERR_INVALID_ARG, "rtt_replica_lift: term " + std::to_string(k) +
                                                        " names a spin twice");
            }
            seen[j] = 1;
            if (ops[f] == 2) {
                row[R[(size_t)j * nb + block[k]]] = 2;
            } else if (ops[f] == 1) {
                for (int c = 0; c < nb; ++c) row[R[(size_t)j * nb + c]] = 1;
            } else {
                for (int g = f0; g <= f; ++g) seen[spins[g]] = 0;
                return rp_fail(ops[f] == 3 ? RTT_ERR_UNSUPPORTED : RTT_ERR_INVALID_ARG,
                               "rtt_replica_lift: only X (1) and Z (2) factors are lifted");
            }
        }
        for (int f = f0; f < f1; ++f) seen[spins[f]] = 0;
        eta_out[k] = coef[k];
    }
    return RTT_OK;
}

rtt_status rtt_tt_plan_create(int32_t length, int32_t chi, int32_t chi_tree, int32_t precision,
                              int32_t n_terms, const uint8_t *ops, const double *eta,
                              int32_t device, rtt_tt_plan *out) {
    if (!out) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_plan_create: out is null");
    *out = nullptr;
    if (length < 2 || chi < 1 || n_terms < 1 || !ops || !eta)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_plan_create: need length >= 2, chi >= 1, "
                                            "n_terms >= 1 and non-null ops, eta");
    if (chi > kMaxChi) return rp_fail(RTT_ERR_UNSUPPORTED, "rtt_tt_plan_create: chi > 16");
    if (precision != RTT_FP64 && precision != RTT_FP32)
        return rp_fail(RTT_ERR_UNSUPPORTED, "rtt_tt_plan_create: precision must be FP64 or FP32");
    if (chi_tree == 0) chi_tree = std::min(2 * chi, kMaxChi);
    if (chi_tree < chi || chi_tree > kMaxChi)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_plan_create: need chi <= chi_tree <= 16");
    for (size_t i = 0; i < (size_t)n_terms * length; ++i)
        if (ops[i] > 2) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_plan_create: string code > 2");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    rtt_tt_plan_s *p = new rtt_tt_plan_s();
    p->device = device;
    p->L = length;
    p->chi = chi;
    p->K = n_terms;
    p->precision = precision;
    p->chi_tree = chi_tree;
    p->cm = std::max(chi, chi_tree);
    p->eta.assign(eta, eta + n_terms);
    p->max_pairs = std::max(1, n_terms / 2);
    p->qsite = q_site_doubles(p->cm);
    const size_t tt = (size_t)length * 2 * chi * chi;
    const size_t ttn = (size_t)length * 2 * chi_tree * chi_tree;
    int n_pairs_total = n_terms;                 // K - 1 tree pairs + the final one
    auto cleanup = [&](cudaError_t err) {
        rtt_tt_plan_destroy(p);
        return rp_fail(err == cudaErrorMemoryAllocation ? RTT_ERR_OOM : RTT_ERR_CUDA,
                       std::string("rtt_tt_plan_create: ") + cudaGetErrorString(err));
    };
    if ((e = cudaMalloc(&p->d_ops, (size_t)n_terms * length)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemcpy(p->d_ops, ops, (size_t)n_terms * length, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(e);
    if (n_terms > 1 && (e = cudaMalloc(&p->d_nodes, (size_t)(n_terms - 1) * ttn * 8)) != cudaSuccess)
        return cleanup(e);
    if ((e = cudaMalloc(&p->d_next, tt * 8)) != cudaSuccess) return cleanup(e);
    const size_t esz = precision == RTT_FP32 ? 4 : 8;
    if ((e = cudaMalloc(&p->d_scratch, (size_t)p->max_pairs * length * p->qsite * esz)) != cudaSuccess)
        return cleanup(e);
    if ((e = cudaMalloc(&p->d_pairs, (size_t)n_pairs_total * sizeof(TTPair))) != cudaSuccess)
        return cleanup(e);
    *out = p;
    return RTT_OK;
}

rtt_status rtt_tt_plan_destroy(rtt_tt_plan p) {
    if (!p) return RTT_OK;
    cudaSetDevice(p->device);
    cudaFree(p->d_ops);
    cudaFree(p->d_nodes);
    cudaFree(p->d_next);
    cudaFree(p->d_scratch);
    cudaFree(p->d_pairs);
    delete p;
    return RTT_OK;
}

rtt_status rtt_tt_power(rtt_tt_plan p, double *phi, double tau, int32_t n_steps, double *log_norm,
                        void *stream) {
    if (!p || !phi || n_steps < 0) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_power: bad arguments");
    if (n_steps == 0) return RTT_OK;
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    if (!p->pairs_valid || p->pairs_phi != phi || p->pairs_tau != tau) {
        std::vector<TTPair> pairs;
        build_pairs(p, phi, tau, pairs);
        // pageable source: staged before the call returns, copied in stream
        // order (after earlier work that read the old table)
        if ((e = cudaMemcpyAsync(p->d_pairs, pairs.data(), pairs.size() * sizeof(TTPair),
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_power: ") + cudaGetErrorString(e));
        p->pairs_phi = phi;
        p->pairs_tau = tau;
        p->pairs_valid = true;
    }
    const size_t tt = (size_t)p->L * 2 * p->chi * p->chi;
    const int nlev = (int)p->level_off.size() - 1;
    const int final_idx = p->level_off.back();
    for (int step = 0; step < n_steps; ++step) {
        for (int l = 0; l < nlev; ++l) {
            const int n = p->level_off[l + 1] - p->level_off[l];
            if ((e = launch_round_any(p->d_pairs + p->level_off[l], n, p->L, p->cm, p->precision,
                                      p->d_scratch, 0, nullptr, st)) != cudaSuccess)
                return rp_fail(RTT_ERR_CUDA, std::string("k_tt_round: ") + cudaGetErrorString(e));
        }
        if ((e = launch_round_any(p->d_pairs + final_idx, 1, p->L, p->cm, p->precision, p->d_scratch, 1,
                                  log_norm ? log_norm + step : nullptr, st)) != cudaSuccess)
            return rp_fail(RTT_ERR_CUDA, std::string("k_tt_round: ") + cudaGetErrorString(e));
        if ((e = cudaMemcpyAsync(phi, p->d_next, tt * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_power: ") + cudaGetErrorString(e));
    }
    return RTT_OK;
}

rtt_status rtt_tt_apply(rtt_tt_plan p, const double *phi, int32_t chi_phi, double *out,
                        double *log_norm, void *stream) {
    if (!p || !phi || !out) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_apply: null pointer");
    if (out == phi) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_apply: out aliases phi");
    if (chi_phi == 0) chi_phi = p->chi;
    if (chi_phi < 1 || chi_phi > p->cm)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_apply: chi_phi must be in [1, max(chi, chi_tree)]");
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    std::vector<TTPair> pairs;
    TTItem root = build_tree(p, term_items(p, phi, chi_phi), pairs);
    TTItem zero = root;
    zero.coef = 0.0;
    pairs.push_back(TTPair{root, zero, out, p->chi});
    p->pairs_valid = false;
    if ((e = run_pairs(p, pairs, log_norm, (cudaStream_t)stream)) != cudaSuccess)
        return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_apply: ") + cudaGetErrorString(e));
    return RTT_OK;
}

rtt_status rtt_tt_sum_round(rtt_tt_plan p, int32_t n, const double *const *tts, int32_t chi_in,
                            const double *coef, double *out, double *log_norm, void *stream) {
    if (!p || !tts || !coef || !out || n < 1)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_sum_round: null pointer or n < 1");
    if (chi_in == 0) chi_in = p->chi;
    if (chi_in < 1 || chi_in > p->cm)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_sum_round: chi_in must be in [1, max(chi, chi_tree)]");
    if (n > p->K)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_sum_round: n exceeds the plan's term count");
    std::vector<TTItem> items(n);
    for (int m = 0; m < n; ++m) {
        if (!tts[m] || tts[m] == out)
            return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_sum_round: null input or out aliases one");
        items[m] = TTItem{tts[m], nullptr, coef[m], chi_in};
    }
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    std::vector<TTPair> pairs;
    TTItem root = build_tree(p, items, pairs);
    TTItem zero = root;
    zero.coef = 0.0;
    pairs.push_back(TTPair{root, zero, out, p->chi});
    p->pairs_valid = false;
    if ((e = run_pairs(p, pairs, log_norm, (cudaStream_t)stream)) != cudaSuccess)
        return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_sum_round: ") + cudaGetErrorString(e));
    return RTT_OK;
}

rtt_status rtt_tt_round_sum(rtt_tt_plan p, const double *a, const uint8_t *ops_a, double coef_a,
                            const double *b, const uint8_t *ops_b, double coef_b, double *out,
                            double *log_norm, void *stream) {
    if (!p || !a || !b || !out) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_round_sum: null pointer");
    if (out == a || out == b) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_round_sum: out aliases an input");
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    TTPair pr{TTItem{a, ops_a, coef_a, p->chi}, TTItem{b, ops_b, coef_b, p->chi}, out, p->chi};
    // the device pair lives in the plan's pair table (slot 0); the power
    // method rebuilds its table on its next call
    p->pairs_valid = false;
    if ((e = cudaMemcpyAsync(p->d_pairs, &pr, sizeof(TTPair), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_round_sum: ") + cudaGetErrorString(e));
    if ((e = launch_round_any(p->d_pairs, 1, p->L, p->cm, p->precision, p->d_scratch, log_norm ? 1 : 0,
                              log_norm,
                              st)) != cudaSuccess)
        return rp_fail(RTT_ERR_CUDA, std::string("k_tt_round: ") + cudaGetErrorString(e));
    return RTT_OK;
}

}  // extern "C"
