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
// Lanes own matrix columns (at most 2 chi <= 32 of them), so a reflector or a
// rotation is one sequential loop per lane and no cross-lane reduction.  All
// arithmetic is FP64: a rounding is a chain of L small dependent
// factorizations, bound by latency rather than arithmetic throughput.
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
};
struct TTPair {
    TTItem a, b;
    double *out;          // padded cores [L][2][chi][chi]
};

rtt_status rp_fail(rtt_status s, const std::string &msg) {
    rtt_set_error(msg);
    return s;
}

// Per-warp shared memory (doubles), CM = compile-time bound on chi.
template <int CM>
struct WarpSmem {
    static constexpr int D2 = 2 * CM, MR = 4 * CM;
    double m[D2][MR];        // sweep 1: columns of the matrix being factored (then Q)
    double v[D2][MR];        // sweep 1: Householder vectors
    double beta[D2];
    double r[D2][D2];        // R factor carried to the next site (row-major)
    double x[2][D2][D2];     // sweep 2: columns being rotated (double-buffered)
    double vv[2][D2][D2];    // sweep 2: accumulated rotations, columns
    double w[D2][CM];        // sweep 2: U S carried to the left, [row][kept column]
    double sig[D2];
    int sel[CM];
};

// Element (b, s, c) of the sum core at site k: block diagonal in the middle,
// [a | b] at the first site, [a ; b] stacked at the last; strings applied.
__device__ __forceinline__ double item_core(const TTItem &it, int L, int chi, int k, int s,
                                            int b, int c) {
    int so = s;
    double sg = 1.0;
    if (it.ops) {
        const uint8_t op = it.ops[k];
        if (op == 1) so = 1 - s;
        else if (op == 2 && s == 1) sg = -1.0;
    }
    if (k == 0) sg *= it.coef;
    return sg * it.tt[(((size_t)k * 2 + so) * chi + b) * chi + c];
}

__device__ __forceinline__ double sum_core(const TTItem &A, const TTItem &B, int L, int chi, int k,
                                           int s, int b, int c) {
    if (k == 0) {                         // left rank 1
        return c < chi ? item_core(A, L, chi, k, s, 0, c) : item_core(B, L, chi, k, s, 0, c - chi);
    }
    if (k == L - 1) {                     // right rank 1
        return b < chi ? item_core(A, L, chi, k, s, b, 0) : item_core(B, L, chi, k, s, b - chi, 0);
    }
    if (b < chi && c < chi) return item_core(A, L, chi, k, s, b, c);
    if (b >= chi && c >= chi) return item_core(B, L, chi, k, s, b - chi, c - chi);
    return 0.0;
}

template <int CM>
__global__ void __launch_bounds__(128) k_tt_round(const TTPair *__restrict__ pairs, int npairs,
                                                  int L, int chi, double *__restrict__ scratch,
                                                  int normalize, double *__restrict__ log_norm) {
    constexpr int D2M = 2 * CM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    if (w >= npairs) return;
    WarpSmem<CM> &S = reinterpret_cast<WarpSmem<CM> *>(smem_raw)[wib];
    const TTPair P = pairs[w];
    const int D2 = 2 * chi;
    const size_t qstride = (size_t)2 * D2M * D2M;            // one site's Q, [row (a,s)][col]
    double *Q = scratch + (size_t)w * L * qstride;

    // ---------------- sweep 1: left to right, Householder QR -----------------
    // R starts as the 1 x 1 identity (left rank 1 at the first site).
    if (lane == 0) S.r[0][0] = 1.0;
    __syncwarp();
    int rl = 1;                                  // rows of R = left rank of M
    for (int k = 0; k < L; ++k) {
        const int dl = (k == 0) ? 1 : D2;        // left bond of the sum core
        const int dr = (k == L - 1) ? 1 : D2;    // right bond
        const int mr = 2 * rl;                   // rows of M, (a, s) -> a * 2 + s
        // M = R x_1 G_k, lanes own columns c < dr
        if (lane < dr) {
            for (int a = 0; a < rl; ++a)
                for (int s = 0; s < 2; ++s) {
                    double acc = 0.0;
                    for (int b = 0; b < dl; ++b) {
                        const double g = sum_core(P.a, P.b, L, chi, k, s, b, lane);
                        acc = fma(S.r[a][b], g, acc);
                    }
                    S.m[lane][a * 2 + s] = acc;
                }
        }
        __syncwarp();
        double *Qk = Q + (size_t)k * qstride;
        if (k == L - 1) {                        // the last core keeps R absorbed
            for (int i = lane; i < mr; i += 32) Qk[(size_t)i * D2M] = S.m[0][i];
            __syncwarp();
            break;
        }
        const int m = min(mr, dr);
        for (int j = 0; j < m; ++j) {
            if (lane == j) {
                double n2 = 0.0;
                for (int i = j; i < mr; ++i) n2 = fma(S.m[j][i], S.m[j][i], n2);
                const double x0 = S.m[j][j];
                double beta = 0.0, alpha = 0.0;
                if (n2 > 0.0) {
                    alpha = x0 >= 0.0 ? -sqrt(n2) : sqrt(n2);
                    const double v0 = x0 - alpha;
                    const double vtv = n2 - x0 * x0 + v0 * v0;
                    beta = vtv > 0.0 ? 2.0 / vtv : 0.0;
                    S.v[j][j] = v0;
                    for (int i = j + 1; i < mr; ++i) S.v[j][i] = S.m[j][i];
                } else {
                    for (int i = j; i < mr; ++i) S.v[j][i] = 0.0;
                    alpha = 0.0;
                }
                S.beta[j] = beta;
                S.m[j][j] = alpha;
                for (int i = j + 1; i < mr; ++i) S.m[j][i] = 0.0;
            }
            __syncwarp();
            if (lane > j && lane < dr) {
                const double beta = S.beta[j];
                double d = 0.0;
                for (int i = j; i < mr; ++i) d = fma(S.v[j][i], S.m[lane][i], d);
                d *= beta;
                for (int i = j; i < mr; ++i) S.m[lane][i] = fma(-d, S.v[j][i], S.m[lane][i]);
            }
            __syncwarp();
        }
        // R (m x dr, upper trapezoidal) for the next site
        if (lane < dr)
            for (int j = 0; j < m; ++j) S.r[j][lane] = (j <= lane) ? S.m[lane][j] : 0.0;
        __syncwarp();
        // Q = H_0 ... H_{m-1} I[:, :m], lanes own columns c < m
        if (lane < m) {
            for (int i = 0; i < mr; ++i) S.m[lane][i] = (i == lane) ? 1.0 : 0.0;
            for (int j = m - 1; j >= 0; --j) {
                const double beta = S.beta[j];
                double d = 0.0;
                for (int i = j; i < mr; ++i) d = fma(S.v[j][i], S.m[lane][i], d);
                d *= beta;
                for (int i = j; i < mr; ++i) S.m[lane][i] = fma(-d, S.v[j][i], S.m[lane][i]);
            }
            for (int i = 0; i < mr; ++i) Qk[(size_t)i * D2M + lane] = S.m[lane][i];
        }
        __syncwarp();
        rl = m;
    }

    // ---------------- sweep 2: right to left, truncated SVD ------------------
    // rank to the left of site k after sweep 1: min(2^k, 2 chi)
    auto rank_left = [&](int k) { return k >= 5 ? D2 : min(1 << k, D2); };
    double *out = P.out;
    // N for site L-1: rows a < r0, columns s (right rank 1)
    int r1 = 1;
    int cur = 0;
    {
        const int r0 = rank_left(L - 1);
        const double *Qk = Q + (size_t)(L - 1) * qstride;
        if (lane < 2)
            for (int a = 0; a < r0; ++a) S.x[0][lane][a] = Qk[(size_t)(a * 2 + lane) * D2M];
        __syncwarp();
    }
    for (int k = L - 1; k >= 1; --k) {
        const int r0 = rank_left(k);
        const int n2 = 2 * r1;                   // columns (s, c) -> s * r1 + c
        // V = I
        if (lane < n2)
            for (int i = 0; i < n2; ++i) S.vv[cur][lane][i] = (i == lane) ? 1.0 : 0.0;
        __syncwarp();
        // Hestenes sweeps with a round-robin tournament (n2 even)
        for (int sweep = 0; sweep < 60; ++sweep) {
            int rotated = 0;
            for (int rnd = 0; rnd < n2 - 1; ++rnd) {
                const int nxt = cur ^ 1;
                if (lane < n2) {
                    // circle method: player 0 fixed, the others rotate
                    const int pos = (lane == 0) ? 0 : ((lane - 1 - rnd + 2 * (n2 - 1)) % (n2 - 1)) + 1;
                    const int ppos = n2 - 1 - pos;
                    const int partner = (ppos == 0) ? 0 : ((ppos - 1 + rnd) % (n2 - 1)) + 1;
                    const int lo = min(lane, partner), hi = max(lane, partner);
                    double a = 0.0, b = 0.0, g = 0.0;
                    for (int i = 0; i < r0; ++i) {
                        const double xl = S.x[cur][lo][i], xh = S.x[cur][hi][i];
                        a = fma(xl, xl, a);
                        b = fma(xh, xh, b);
                        g = fma(xl, xh, g);
                    }
                    double c = 1.0, sn = 0.0;
                    if (g != 0.0 && fabs(g) > 2.220446049250313e-16 * sqrt(a * b)) {
                        const double zeta = (b - a) / (2.0 * g);
                        // smaller root of t^2 + 2 zeta t - 1 = 0; 1/(2 zeta) once zeta^2 would overflow
                        const double t = fabs(zeta) > 1e150
                                             ? 0.5 / zeta
                                             : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = c * t;
                        rotated = 1;
                    }
                    // lo' = c lo - s hi, hi' = s lo + c hi
                    const bool am_lo = (lane == lo);
                    for (int i = 0; i < r0; ++i) {
                        const double xl = S.x[cur][lo][i], xh = S.x[cur][hi][i];
                        S.x[nxt][lane][i] = am_lo ? (c * xl - sn * xh) : (sn * xl + c * xh);
                    }
                    for (int i = 0; i < n2; ++i) {
                        const double vl = S.vv[cur][lo][i], vh = S.vv[cur][hi][i];
                        S.vv[nxt][lane][i] = am_lo ? (c * vl - sn * vh) : (sn * vl + c * vh);
                    }
                }
                __syncwarp();
                cur ^= 1;
            }
            if (!__any_sync(0xffffffffu, rotated)) break;
        }
        // singular values and the kept columns, largest first (ties by index)
        if (lane < n2) {
            double s2 = 0.0;
            for (int i = 0; i < r0; ++i) s2 = fma(S.x[cur][lane][i], S.x[cur][lane][i], s2);
            S.sig[lane] = sqrt(s2);
        }
        __syncwarp();
        const int t = min(chi, min(r0, n2));
        if (lane < n2) {
            int rank = 0;
            for (int j = 0; j < n2; ++j)
                rank += (S.sig[j] > S.sig[lane]) || (S.sig[j] == S.sig[lane] && j < lane);
            if (rank < t) S.sel[rank] = lane;
        }
        __syncwarp();
        // output core k: rows i < t are columns sel[i] of V, reshaped (s, c)
        for (int e = lane; e < 2 * chi * chi; e += 32) {
            const int s = e / (chi * chi), i = (e / chi) % chi, c = e % chi;
            double val = 0.0;
            if (i < t && c < r1) val = S.vv[cur][S.sel[i]][s * r1 + c];
            out[(size_t)k * 2 * chi * chi + e] = val;
        }
        // U S for the site to the left: w[row][i] = rotated column sel[i]
        for (int e = lane; e < r0 * t; e += 32) {
            const int row = e / t, i = e % t;
            S.w[row][i] = S.x[cur][S.sel[i]][row];
        }
        __syncwarp();
        // next N: Q_{k-1} (r0' x 2 x r0) x_3 w (r0 x t), columns (s, i) -> s * t + i
        const int rp = rank_left(k - 1);
        const double *Qp = Q + (size_t)(k - 1) * qstride;
        const int nn = 2 * t;
        if (lane < nn) {
            const int s = lane / t, i = lane % t;
            for (int a = 0; a < rp; ++a) {
                double acc = 0.0;
                for (int b = 0; b < r0; ++b) acc = fma(Qp[(size_t)(a * 2 + s) * D2M + b], S.w[b][i], acc);
                S.x[cur][lane][a] = acc;
            }
        }
        __syncwarp();
        r1 = t;
    }
    // first core: 1 x 2 x r1, optionally scaled to unit norm
    double scale = 1.0;
    if (normalize) {
        double s2 = 0.0;
        for (int j = 0; j < 2 * r1; ++j) s2 = fma(S.x[cur][j][0], S.x[cur][j][0], s2);
        const double nrm = sqrt(s2);
        scale = 1.0 / nrm;
        if (lane == 0 && log_norm) log_norm[w] = log(nrm);
    }
    for (int e = lane; e < 2 * chi * chi; e += 32) {
        const int s = e / (chi * chi), i = (e / chi) % chi, c = e % chi;
        double val = 0.0;
        if (i == 0 && c < r1) val = S.x[cur][s * r1 + c][0] * scale;
        out[e] = val;
    }
}

template <int CM>
constexpr int warps_per_cta() {
    return CM <= 4 ? 4 : (CM <= 8 ? 2 : 1);
}

template <int CM>
cudaError_t launch_round(const TTPair *pairs, int npairs, int L, int chi, double *scratch,
                         int normalize, double *log_norm, cudaStream_t st) {
    constexpr int wpc = warps_per_cta<CM>();
    const size_t smem = sizeof(WarpSmem<CM>) * wpc;
    // per device and cheap: set on every launch
    cudaError_t e = cudaFuncSetAttribute(k_tt_round<CM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (npairs + wpc - 1) / wpc;
    k_tt_round<CM><<<blocks, 32 * wpc, smem, st>>>(pairs, npairs, L, chi, scratch, normalize,
                                                   log_norm);
    return cudaGetLastError();
}

cudaError_t launch_round_any(const TTPair *pairs, int npairs, int L, int chi, double *scratch,
                             int normalize, double *log_norm, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    if (chi <= 4) return launch_round<4>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
    if (chi <= 8) return launch_round<8>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
    return launch_round<16>(pairs, npairs, L, chi, scratch, normalize, log_norm, st);
}

}  // namespace

// ----------------------------------------------------------------------------
// Plan
// ----------------------------------------------------------------------------
struct rtt_tt_plan_s {
    int device = 0, L = 0, chi = 0, K = 0;
    std::vector<double> eta;
    uint8_t *d_ops = nullptr;     // [K][L]
    double *d_nodes = nullptr;    // [K-1][L][2][chi][chi] tree node TTs
    double *d_next = nullptr;     // [L][2][chi][chi]
    double *d_scratch = nullptr;  // [max pairs][L][2 (2chi)^2] (padded to the kernel's bound)
    TTPair *d_pairs = nullptr;    // the tree's pairs, level by level, then the final pair
    std::vector<int> level_off;   // pairs of level l: [level_off[l], level_off[l+1])
    int max_pairs = 1;
    size_t qsite = 0;             // doubles of one site's Q in the scratch
    const double *pairs_phi = nullptr;  // phi and tau the device pairs were built for
    double pairs_tau = 0.0;
    bool pairs_valid = false;
};

namespace {

size_t q_site_doubles(int chi) {
    const int cm = chi <= 4 ? 4 : (chi <= 8 ? 8 : 16);
    return (size_t)2 * (2 * cm) * (2 * cm);
}

// Pairs of the tree over `items` (two by two, an odd last item passes up),
// level by level, node outputs in the plan's node buffers in creation order;
// appends to `pairs`, sets the plan's level offsets and returns the root.
TTItem build_tree(rtt_tt_plan_s *p, std::vector<TTItem> items, std::vector<TTPair> &pairs) {
    const size_t tt = (size_t)p->L * 2 * p->chi * p->chi;
    pairs.clear();
    p->level_off.assign(1, 0);
    int node = 0;
    while (items.size() > 1) {
        std::vector<TTItem> nxt;
        for (size_t i = 0; i + 1 < items.size(); i += 2) {
            double *o = p->d_nodes + (size_t)node++ * tt;
            pairs.push_back(TTPair{items[i], items[i + 1], o});
            nxt.push_back(TTItem{o, nullptr, 1.0});
        }
        if (items.size() % 2) nxt.push_back(items.back());
        items.swap(nxt);
        p->level_off.push_back((int)pairs.size());
    }
    return items[0];
}

std::vector<TTItem> term_items(rtt_tt_plan_s *p, const double *phi) {
    std::vector<TTItem> items(p->K);
    for (int k = 0; k < p->K; ++k) items[k] = TTItem{phi, p->d_ops + (size_t)k * p->L, p->eta[k]};
    return items;
}

// (1 - tau H-bar): the tree's root S, then phi - tau S into the plan's next buffer.
void build_pairs(rtt_tt_plan_s *p, const double *phi, double tau, std::vector<TTPair> &pairs) {
    TTItem s = build_tree(p, term_items(p, phi), pairs);
    s.coef *= -tau;
    pairs.push_back(TTPair{TTItem{phi, nullptr, 1.0}, s, p->d_next});
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
        if ((e = launch_round_any(p->d_pairs + p->level_off[l], n, p->L, p->chi, p->d_scratch, 0,
                                  nullptr, st)) != cudaSuccess)
            return e;
    }
    return launch_round_any(p->d_pairs + p->level_off.back(), 1, p->L, p->chi, p->d_scratch, 1,
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

rtt_status rtt_tt_plan_create(int32_t length, int32_t chi, int32_t n_terms, const uint8_t *ops,
                              const double *eta, int32_t device, rtt_tt_plan *out) {
    if (!out) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_plan_create: out is null");
    *out = nullptr;
    if (length < 2 || chi < 1 || n_terms < 1 || !ops || !eta)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_plan_create: need length >= 2, chi >= 1, "
                                            "n_terms >= 1 and non-null ops, eta");
    if (chi > kMaxChi) return rp_fail(RTT_ERR_UNSUPPORTED, "rtt_tt_plan_create: chi > 16");
    for (size_t i = 0; i < (size_t)n_terms * length; ++i)
        if (ops[i] > 2) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_plan_create: string code > 2");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    rtt_tt_plan_s *p = new rtt_tt_plan_s();
    p->device = device;
    p->L = length;
    p->chi = chi;
    p->K = n_terms;
    p->eta.assign(eta, eta + n_terms);
    p->max_pairs = std::max(1, n_terms / 2);
    p->qsite = q_site_doubles(chi);
    const size_t tt = (size_t)length * 2 * chi * chi;
    int n_pairs_total = n_terms;                 // K - 1 tree pairs + the final one
    auto cleanup = [&](cudaError_t err) {
        rtt_tt_plan_destroy(p);
        return rp_fail(err == cudaErrorMemoryAllocation ? RTT_ERR_OOM : RTT_ERR_CUDA,
                       std::string("rtt_tt_plan_create: ") + cudaGetErrorString(err));
    };
    if ((e = cudaMalloc(&p->d_ops, (size_t)n_terms * length)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMemcpy(p->d_ops, ops, (size_t)n_terms * length, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(e);
    if (n_terms > 1 && (e = cudaMalloc(&p->d_nodes, (size_t)(n_terms - 1) * tt * 8)) != cudaSuccess)
        return cleanup(e);
    if ((e = cudaMalloc(&p->d_next, tt * 8)) != cudaSuccess) return cleanup(e);
    if ((e = cudaMalloc(&p->d_scratch, (size_t)p->max_pairs * length * p->qsite * 8)) != cudaSuccess)
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
            if ((e = launch_round_any(p->d_pairs + p->level_off[l], n, p->L, p->chi, p->d_scratch,
                                      0, nullptr, st)) != cudaSuccess)
                return rp_fail(RTT_ERR_CUDA, std::string("k_tt_round: ") + cudaGetErrorString(e));
        }
        if ((e = launch_round_any(p->d_pairs + final_idx, 1, p->L, p->chi, p->d_scratch, 1,
                                  log_norm ? log_norm + step : nullptr, st)) != cudaSuccess)
            return rp_fail(RTT_ERR_CUDA, std::string("k_tt_round: ") + cudaGetErrorString(e));
        if ((e = cudaMemcpyAsync(phi, p->d_next, tt * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_power: ") + cudaGetErrorString(e));
    }
    return RTT_OK;
}

rtt_status rtt_tt_apply(rtt_tt_plan p, const double *phi, double *out, double *log_norm,
                        void *stream) {
    if (!p || !phi || !out) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_apply: null pointer");
    if (out == phi) return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_apply: out aliases phi");
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    std::vector<TTPair> pairs;
    TTItem root = build_tree(p, term_items(p, phi), pairs);
    TTItem zero = root;
    zero.coef = 0.0;
    pairs.push_back(TTPair{root, zero, out});
    p->pairs_valid = false;
    if ((e = run_pairs(p, pairs, log_norm, (cudaStream_t)stream)) != cudaSuccess)
        return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_apply: ") + cudaGetErrorString(e));
    return RTT_OK;
}

rtt_status rtt_tt_sum_round(rtt_tt_plan p, int32_t n, const double *const *tts, const double *coef,
                            double *out, double *log_norm, void *stream) {
    if (!p || !tts || !coef || !out || n < 1)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_sum_round: null pointer or n < 1");
    if (n > p->K)
        return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_sum_round: n exceeds the plan's term count");
    std::vector<TTItem> items(n);
    for (int m = 0; m < n; ++m) {
        if (!tts[m] || tts[m] == out)
            return rp_fail(RTT_ERR_INVALID_ARG, "rtt_tt_sum_round: null input or out aliases one");
        items[m] = TTItem{tts[m], nullptr, coef[m]};
    }
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return rp_fail(RTT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    std::vector<TTPair> pairs;
    TTItem root = build_tree(p, items, pairs);
    TTItem zero = root;
    zero.coef = 0.0;
    pairs.push_back(TTPair{root, zero, out});
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
    TTPair pr{TTItem{a, ops_a, coef_a}, TTItem{b, ops_b, coef_b}, out};
    // the device pair lives in the plan's pair table (slot 0); the power
    // method rebuilds its table on its next call
    p->pairs_valid = false;
    if ((e = cudaMemcpyAsync(p->d_pairs, &pr, sizeof(TTPair), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return rp_fail(RTT_ERR_CUDA, std::string("rtt_tt_round_sum: ") + cudaGetErrorString(e));
    if ((e = launch_round_any(p->d_pairs, 1, p->L, p->chi, p->d_scratch, log_norm ? 1 : 0, log_norm,
                              st)) != cudaSuccess)
        return rp_fail(RTT_ERR_CUDA, std::string("k_tt_round: ") + cudaGetErrorString(e));
    return RTT_OK;
}

}  // extern "C"
