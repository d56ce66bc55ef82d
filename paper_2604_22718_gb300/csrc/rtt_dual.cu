// rtt_dual.cu -- host parts of dual Monte Carlo (Sec. 3.3): the direct sum of
// RTTs (a linear combination of RTT states as one RTT) and the small
// generalized eigenproblem H~ c = lambda S~ c (Eq. gen_eig2).  No device code.
#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "rtt_internal.cuh"

namespace {

rtt_status dual_fail(rtt_status s, const std::string &msg) {
    rtt_set_error(msg);
    return s;
}

typedef std::complex<double> cd;

// Solve S X = H (n x n, row-major) by LU with partial pivoting; false if singular.
bool lu_solve(int n, std::vector<double> S, const std::vector<double> &H, std::vector<double> &X) {
    std::vector<int> piv(n);
    double smax = 0.0;
    for (double v : S) smax = std::max(smax, std::fabs(v));
    if (!(smax > 0.0) || !std::isfinite(smax)) return false;
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(S[i * n + k]) > std::fabs(S[p * n + k])) p = i;
        if (std::fabs(S[p * n + k]) <= 1e-14 * smax) return false;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(S[k * n + j], S[p * n + j]);
        for (int i = k + 1; i < n; ++i) {
            const double f = S[i * n + k] / S[k * n + k];
            S[i * n + k] = f;
            for (int j = k + 1; j < n; ++j) S[i * n + j] -= f * S[k * n + j];
        }
    }
    X = H;
    for (int col = 0; col < n; ++col) {
        std::vector<double> y(n);
        for (int i = 0; i < n; ++i) y[i] = X[i * n + col];
        for (int k = 0; k < n; ++k) std::swap(y[k], y[piv[k]]);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) y[i] -= S[i * n + j] * y[j];
        for (int i = n - 1; i >= 0; --i) {
            for (int j = i + 1; j < n; ++j) y[i] -= S[i * n + j] * y[j];
            y[i] /= S[i * n + i];
        }
        for (int i = 0; i < n; ++i) X[i * n + col] = y[i];
    }
    return true;
}

// Eigenvalues of a general n x n matrix: Householder reduction to upper
// Hessenberg form, then single-shift QR in complex arithmetic with Givens
// rotations, Wilkinson shifts and deflation of negligible subdiagonals.
bool eigenvalues(int n, const std::vector<double> &A, std::vector<cd> &w) {
    std::vector<cd> H(n * n);
    for (int i = 0; i < n * n; ++i) H[i] = A[i];
    for (int k = 0; k + 2 < n; ++k) {  // Householder: zero H[k+2.., k]
        double alpha = 0.0;
        for (int i = k + 1; i < n; ++i) alpha += std::norm(H[i * n + k]);
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        std::vector<cd> v(n, 0.0);
        const cd x0 = H[(k + 1) * n + k];
        const cd phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0);
        v[k + 1] = x0 + phase * alpha;
        for (int i = k + 2; i < n; ++i) v[i] = H[i * n + k];
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
        if (vn == 0.0) continue;
        // H <- (I - 2 v v^*/|v|^2) H (I - 2 v v^*/|v|^2)
        for (int j = 0; j < n; ++j) {
            cd d = 0.0;
            for (int i = k + 1; i < n; ++i) d += std::conj(v[i]) * H[i * n + j];
            d *= 2.0 / vn;
            for (int i = k + 1; i < n; ++i) H[i * n + j] -= v[i] * d;
        }
        for (int i = 0; i < n; ++i) {
            cd d = 0.0;
            for (int j = k + 1; j < n; ++j) d += H[i * n + j] * v[j];
            d *= 2.0 / vn;
            for (int j = k + 1; j < n; ++j) H[i * n + j] -= d * std::conj(v[j]);
        }
    }
    double scale = 0.0;
    for (const cd &z : H) scale = std::max(scale, std::abs(z));
    if (!std::isfinite(scale)) return false;
    w.assign(n, 0.0);
    int hi = n - 1, iter = 0;
    while (hi >= 0) {
        if (hi == 0) {
            w[0] = H[0];
            break;
        }
        // find the active block [lo, hi]
        int lo = hi;
        while (lo > 0) {
            const double sub = std::abs(H[lo * n + lo - 1]);
            const double diag = std::abs(H[lo * n + lo]) + std::abs(H[(lo - 1) * n + lo - 1]);
            if (sub <= 1e-15 * (diag > 0.0 ? diag : scale)) {
                H[lo * n + lo - 1] = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            w[hi] = H[hi * n + hi];
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 200 * n) return false;
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to H[hi][hi]
        const cd a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
        const cd c = H[hi * n + hi - 1], d = H[hi * n + hi];
        const cd tr = a + d, det = a * d - b * c;
        const cd disc = std::sqrt(tr * tr - 4.0 * det);
        const cd l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        cd mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        if (iter % 11 == 10) mu += cd(0.75 * std::abs(H[hi * n + hi - 1]), 0.0);  // exceptional
        // QR step on the block: H - mu I = QR, H <- RQ + mu I (Givens)
        for (int i = lo; i <= hi; ++i) H[i * n + i] -= mu;
        std::vector<cd> cs(hi - lo), sn(hi - lo);
        for (int k = lo; k < hi; ++k) {
            const cd x = H[k * n + k], y = H[(k + 1) * n + k];
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            cd cc = 1.0, ss = 0.0;
            if (r > 0.0) {
                cc = x / r;
                ss = y / r;
            }
            cs[k - lo] = cc;
            sn[k - lo] = ss;
            for (int j = k; j < n; ++j) {  // rows k, k+1 <- G^* rows
                const cd u = H[k * n + j], t = H[(k + 1) * n + j];
                H[k * n + j] = std::conj(cc) * u + std::conj(ss) * t;
                H[(k + 1) * n + j] = -ss * u + cc * t;
            }
        }
        for (int k = lo; k < hi; ++k) {  // columns k, k+1 <- columns G
            const cd cc = cs[k - lo], ss = sn[k - lo];
            for (int i = 0; i <= std::min(hi, k + 2); ++i) {
                const cd u = H[i * n + k], t = H[i * n + k + 1];
                H[i * n + k] = u * cc + t * ss;
                H[i * n + k + 1] = -u * std::conj(ss) + t * std::conj(cc);
            }
        }
        for (int i = lo; i <= hi; ++i) H[i * n + i] += mu;
    }
    return true;
}

}  // namespace

extern "C" rtt_status rtt_create_sum(const rtt_desc *descs, int32_t M, const double *coef,
                                     rtt_handle *out) {
    rtt_set_error("");
    if (!descs || !coef || !out || M < 1)
        return dual_fail(RTT_ERR_INVALID_ARG, "rtt_create_sum: null argument or M < 1");
    *out = nullptr;
    const rtt_desc &d0 = descs[0];
    if (d0.n_spins < 1 || d0.length < 1 || !d0.path)
        return dual_fail(RTT_ERR_INVALID_ARG, "rtt_create_sum: bad first description");
    int64_t chi = 0;
    for (int m = 0; m < M; ++m) {
        const rtt_desc &d = descs[m];
        if (!d.tensors || !d.b_left || !d.b_right || !d.path || d.chi < 1)
            return dual_fail(RTT_ERR_INVALID_ARG, "rtt_create_sum: incomplete description");
        if (d.n_spins != d0.n_spins || d.length != d0.length || d.n_bonds != d0.n_bonds ||
            d.J != d0.J || d.h != d0.h)
            return dual_fail(RTT_ERR_INVALID_ARG,
                             "rtt_create_sum: descriptions differ in N, L, bonds, J or h");
        for (int k = 0; k < d.length; ++k)
            if (d.path[k] != d0.path[k])
                return dual_fail(RTT_ERR_INVALID_ARG, "rtt_create_sum: paths differ");
        for (int t = 0; t < 2 * d.n_bonds; ++t)
            if (!d.bonds || !d0.bonds || d.bonds[t] != d0.bonds[t])
                return dual_fail(RTT_ERR_INVALID_ARG, "rtt_create_sum: bond lists differ");
        if (!std::isfinite(coef[m]))
            return dual_fail(RTT_ERR_NUMERIC, "rtt_create_sum: non-finite coefficient");
        chi += d.chi;
    }
    if (chi > 256) return dual_fail(RTT_ERR_UNSUPPORTED, "rtt_create_sum: summed chi above 256");
    const int L = d0.length, X = (int)chi;
    std::vector<double> t((size_t)L * 2 * X * X, 0.0), bl(X, 0.0), br(X, 0.0);
    int off = 0;
    for (int m = 0; m < M; ++m) {
        const rtt_desc &d = descs[m];
        const int x = d.chi;
        for (int k = 0; k < L; ++k)
            for (int sp = 0; sp < 2; ++sp)
                for (int a = 0; a < x; ++a)
                    for (int b = 0; b < x; ++b)
                        t[(((size_t)k * 2 + sp) * X + off + a) * X + off + b] =
                            d.tensors[(((size_t)k * 2 + sp) * x + a) * x + b];
        for (int a = 0; a < x; ++a) {
            bl[off + a] = coef[m] * d.b_left[a];
            br[off + a] = d.b_right[a];
        }
        off += x;
    }
    rtt_desc sum = d0;
    sum.chi = X;
    sum.tensors = t.data();
    sum.b_left = bl.data();
    sum.b_right = br.data();
    return rtt_create(&sum, out);
}

extern "C" rtt_status rtt_dual_solve(int32_t M, const double *Ht, const double *St, double *eig_re,
                                     double *eig_im, double *c0) {
    rtt_set_error("");
    if (M < 1 || M > 8 || !Ht || !St || !eig_re || !eig_im)
        return dual_fail(RTT_ERR_INVALID_ARG, "rtt_dual_solve: bad arguments (1 <= M <= 8)");
    const int n = M;
    std::vector<double> S(St, St + n * n), H(Ht, Ht + n * n), A;
    for (int i = 0; i < n * n; ++i)
        if (!std::isfinite(S[i]) || !std::isfinite(H[i]))
            return dual_fail(RTT_ERR_NUMERIC, "rtt_dual_solve: non-finite matrix entry");
    if (!lu_solve(n, S, H, A)) return dual_fail(RTT_ERR_NUMERIC, "rtt_dual_solve: S~ is singular");
    std::vector<cd> w;
    if (!eigenvalues(n, A, w)) return dual_fail(RTT_ERR_NUMERIC, "rtt_dual_solve: QR did not converge");
    std::sort(w.begin(), w.end(), [](const cd &x, const cd &y) {
        return x.real() < y.real() || (x.real() == y.real() && x.imag() < y.imag());
    });
    double wmax = 0.0;
    for (int i = 0; i < n; ++i) {
        eig_re[i] = w[i].real();
        eig_im[i] = w[i].imag();
        wmax = std::max(wmax, std::abs(w[i]));
    }
    if (!c0) return RTT_OK;
    for (int i = 0; i < n; ++i) c0[i] = NAN;
    if (std::fabs(w[0].imag()) > 1e-9 * (wmax > 0.0 ? wmax : 1.0)) return RTT_OK;
    // inverse iteration on A - lambda0 I (lambda0 nudged off exact singularity)
    const double lam = w[0].real() + 1e-10 * (wmax > 0.0 ? wmax : 1.0);
    std::vector<double> B(A), x(n, 1.0), y;
    for (int i = 0; i < n; ++i) B[i * n + i] -= lam;
    for (int it = 0; it < 4; ++it) {
        std::vector<double> rhs(n * n, 0.0);
        for (int i = 0; i < n; ++i) rhs[i * n] = x[i];
        std::vector<double> sol;
        if (!lu_solve(n, B, rhs, sol)) break;  // exactly singular: x is already the vector
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) nrm = std::max(nrm, std::fabs(sol[i * n]));
        if (!(nrm > 0.0) || !std::isfinite(nrm)) break;
        for (int i = 0; i < n; ++i) x[i] = sol[i * n] / nrm;
    }
    double q = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) q += x[i] * S[i * n + j] * x[j];
    if (q != 0.0 && std::isfinite(q)) {
        const double f = 1.0 / std::sqrt(std::fabs(q));
        for (int i = 0; i < n; ++i) x[i] *= f;
    }
    int k = 0;
    for (int i = 1; i < n; ++i)
        if (std::fabs(x[i]) > std::fabs(x[k])) k = i;
    const double sgn = x[k] < 0 ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) c0[i] = sgn * x[i];
    return RTT_OK;
}

// Eq. Gram-Schmid: row m of T holds 1 at m and -<psi^m / psi^a>_{P^a} =
// -S~[a][m] at every a < m (a = 0 only when first_only), so psi' = T psi.
extern "C" rtt_status rtt_dual_gram_schmidt(int32_t M, const double *St, int32_t first_only,
                                            double *T) {
    rtt_set_error("");
    if (M < 1 || M > 8 || !St || !T)
        return dual_fail(RTT_ERR_INVALID_ARG, "rtt_dual_gram_schmidt: bad arguments (1 <= M <= 8)");
    // every entry of S~ that T uses is checked before T is written, so an
    // error leaves the caller's T untouched
    for (int m = 0; m < M; ++m)
        for (int a = 0; a < m; ++a)
            if ((!first_only || a == 0) && !std::isfinite(St[a * M + m]))
                return dual_fail(RTT_ERR_NUMERIC, "rtt_dual_gram_schmidt: non-finite S~");
    for (int m = 0; m < M; ++m)
        for (int a = 0; a < M; ++a) {
            double v = a == m ? 1.0 : 0.0;
            if (a < m && (!first_only || a == 0)) v = -St[a * M + m];
            T[m * M + a] = v;
        }
    return RTT_OK;
}

// psi' = T psi and sum_m c'_m psi'^m = sum_a c_a psi^a give c = T^T c',
// summed over m in increasing order.
extern "C" rtt_status rtt_dual_back_transform(int32_t M, const double *T, const double *c_prime,
                                              double *c) {
    rtt_set_error("");
    if (M < 1 || M > 8 || !T || !c_prime || !c || c == c_prime)
        return dual_fail(RTT_ERR_INVALID_ARG, "rtt_dual_back_transform: bad arguments (1 <= M <= 8)");
    for (int a = 0; a < M; ++a) {
        double acc = 0.0;
        for (int m = 0; m < M; ++m) acc += T[m * M + a] * c_prime[m];
        c[a] = acc;
    }
    return RTT_OK;
}
