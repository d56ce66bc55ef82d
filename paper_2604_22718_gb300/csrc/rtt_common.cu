// rtt_common.cu -- kernels shared by every precision: the local-energy
// reduction (Sec. 3.3 / Sec. 4 Eq. ising-model), the Metropolis uniforms, and
// the FP64 trace statistics behind rtt_observables (V-score, Sec. 4.3).
#include <math_constants.h>

#include "rtt_internal.cuh"

namespace {

// One thread per chain.  rows_* [B][N+1]: entry j < N is psi(s^(q[j])),
// entry N is psi(s).  ratios are summed in increasing spin index.
__global__ void k_eloc_reduce(const uint8_t *__restrict__ spins, int64_t B, int N,
                              const int32_t *__restrict__ pos, const int32_t *__restrict__ bonds,
                              int n_bonds, double J, double h,
                              const double *__restrict__ rows_mant,
                              const int64_t *__restrict__ rows_exp, double *__restrict__ e_loc,
                              double *__restrict__ ratios) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    const double *rm = rows_mant + c * (N + 1);
    const int64_t *re = rows_exp + c * (N + 1);
    const uint8_t *s = spins + c * N;
    const double m0 = rm[N];
    const int64_t e0 = re[N];
    if (m0 == 0.0 || !isfinite(m0)) {
        e_loc[c] = CUDART_NAN;
        if (ratios)
            for (int i = 0; i < N; ++i) ratios[c * N + i] = CUDART_NAN;
        return;
    }
    int64_t zz = 0;
    for (int b = 0; b < n_bonds; ++b) {
        const int zi = 1 - 2 * (int)s[bonds[2 * b]];
        const int zj = 1 - 2 * (int)s[bonds[2 * b + 1]];
        zz += zi * zj;
    }
    double sum = 0.0;
    for (int i = 0; i < N; ++i) {
        const int j = pos[i];
        const double ratio = ldexp(rm[j] / m0, (int)(re[j] - e0));
        if (ratios) ratios[c * N + i] = ratio;
        sum += ratio;
    }
    e_loc[c] = J * (double)zz - h * sum;
}

// Mixed local energy of dual Monte Carlo: rows of handle b, amplitude of a.
// Ratios ldexp(mant_b / mant_a, exp_b - exp_a); field term in increasing spin
// index; E = (J zz) r0 - h sum (the FP64 oracle's order).
__global__ void k_mixed_reduce(const uint8_t *__restrict__ spins, int64_t B, int N,
                               const int32_t *__restrict__ pos, const int32_t *__restrict__ bonds,
                               int n_bonds, double J, double h,
                               const double *__restrict__ rows_mant,
                               const int64_t *__restrict__ rows_exp,
                               const rtt_chain_state *__restrict__ amp_a,
                               double *__restrict__ e_mixed, double *__restrict__ ratio) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    const double *rm = rows_mant + c * (N + 1);
    const int64_t *re = rows_exp + c * (N + 1);
    const uint8_t *s = spins + c * N;
    const double ma = amp_a[c].mant;
    const int64_t ea = amp_a[c].exp2;
    if (ma == 0.0 || !isfinite(ma)) {
        if (e_mixed) e_mixed[c] = CUDART_NAN;
        if (ratio) ratio[c] = CUDART_NAN;
        return;
    }
    const double r0 = ldexp(rm[N] / ma, (int)(re[N] - ea));
    double sum = 0.0;
    for (int i = 0; i < N; ++i) {
        const int j = pos[i];
        sum += ldexp(rm[j] / ma, (int)(re[j] - ea));
    }
    int64_t zz = 0;
    for (int b = 0; b < n_bonds; ++b) {
        const int zi = 1 - 2 * (int)s[bonds[2 * b]];
        const int zj = 1 - 2 * (int)s[bonds[2 * b + 1]];
        zz += zi * zj;
    }
    if (e_mixed) e_mixed[c] = J * (double)zz * r0 - h * sum;
    if (ratio) ratio[c] = r0;
}

__global__ void k_uniforms(uint64_t seed, int64_t n, const uint64_t *__restrict__ ctr,
                           double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    out[t] = rttd::mcmc_uniform(seed, ctr[3 * t], ctr[3 * t + 1], ctr[3 * t + 2]);
}

__global__ void k_chain_means(const double *__restrict__ x, int T, int64_t B,
                              double *__restrict__ cm) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += x[(size_t)t * B + c];
    cm[c] = s / (double)T;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
        for (int o = 16; o >= 1; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    return r;
}

// acc[l] += sum_c (1/(T-t)) sum_s d_{s,c} d_{s+t,c},  t = lag0 + l (blockIdx.y)
__global__ void k_lag_sums(const double *__restrict__ x, const double *__restrict__ cm, int T,
                           int64_t B, int lag0, double *__restrict__ acc) {
    const int t = lag0 + (int)blockIdx.y;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (c < B && t < T) {
        const double m = cm[c];
        for (int s = 0; s + t < T; ++s)
            v = fma(x[(size_t)s * B + c] - m, x[(size_t)(s + t) * B + c] - m, v);
        v /= (double)(T - t);
    }
    v = block_sum(v);
    if (threadIdx.x == 0) atomicAdd(acc + blockIdx.y, v);
}

// acc[0] += sum (bm - mean), acc[1] += sum (bm - mean)^2 over bins of length lb
__global__ void k_bin_moments(const double *__restrict__ x, int T, int64_t B, int lb, double mean,
                              double *__restrict__ acc) {
    const int nb = T / lb;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0, d2 = 0.0;
    if (g < (int64_t)nb * B) {
        const int b = (int)(g / B);
        const int64_t c = g % B;
        double s = 0.0;
        for (int t = b * lb; t < (b + 1) * lb; ++t) s += x[(size_t)t * B + c];
        d = s / (double)lb - mean;
        d2 = d * d;
    }
    d = block_sum(d);
    d2 = block_sum(d2);
    if (threadIdx.x == 0) {
        atomicAdd(acc, d);
        atomicAdd(acc + 1, d2);
    }
}

__global__ void k_sum_i64(const int64_t *__restrict__ x, int64_t n, unsigned long long *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long v = (i < n) ? x[i] : 0;
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t eloc_reduce(const uint8_t *spins, int64_t B, int N, const int32_t *pos,
                        const int32_t *bonds, int n_bonds, double J, double h,
                        const double *rows_mant, const int64_t *rows_exp, double *e_loc,
                        double *ratios, cudaStream_t st) {
    k_eloc_reduce<<<nblk(B, 128), 128, 0, st>>>(spins, B, N, pos, bonds, n_bonds, J, h, rows_mant,
                                                 rows_exp, e_loc, ratios);
    return cudaGetLastError();
}

cudaError_t mixed_reduce(const uint8_t *spins, int64_t B, int N, const int32_t *pos,
                         const int32_t *bonds, int n_bonds, double J, double h,
                         const double *rows_mant, const int64_t *rows_exp,
                         const rtt_chain_state *amp_a, double *e_mixed, double *ratio,
                         cudaStream_t st) {
    k_mixed_reduce<<<nblk(B, 128), 128, 0, st>>>(spins, B, N, pos, bonds, n_bonds, J, h, rows_mant,
                                                  rows_exp, amp_a, e_mixed, ratio);
    return cudaGetLastError();
}

cudaError_t launch_uniforms(uint64_t seed, int64_t n, const uint64_t *ctr, double *out,
                            cudaStream_t st) {
    k_uniforms<<<nblk(n, 256), 256, 0, st>>>(seed, n, ctr, out);
    return cudaGetLastError();
}

cudaError_t stats_chain_means(const double *x, int T, int64_t B, double *cm, cudaStream_t st) {
    k_chain_means<<<nblk(B, 256), 256, 0, st>>>(x, T, B, cm);
    return cudaGetLastError();
}

cudaError_t stats_lag_sums(const double *x, const double *cm, int T, int64_t B, int lag0, int nlag,
                           double *acc, cudaStream_t st) {
    dim3 grid(nblk(B, 256), (unsigned)nlag);
    k_lag_sums<<<grid, 256, 0, st>>>(x, cm, T, B, lag0, acc);
    return cudaGetLastError();
}

cudaError_t stats_bin_moments(const double *x, int T, int64_t B, int lb, double mean, double *acc,
                              cudaStream_t st) {
    const int64_t n = (int64_t)(T / lb) * B;
    k_bin_moments<<<nblk(n > 0 ? n : 1, 256), 256, 0, st>>>(x, T, B, lb, mean, acc);
    return cudaGetLastError();
}

cudaError_t stats_sum_i64(const int64_t *x, int64_t n, unsigned long long *out, cudaStream_t st) {
    k_sum_i64<<<nblk(n > 0 ? n : 1, 256), 256, 0, st>>>(x, n, out);
    return cudaGetLastError();
}
