// rtt_made.cu -- learned independence proposal: a MADE (masked autoregressive
// MLP, Germain et al., ICML 2015) trained and sampled by this library's own
// kernels, and the independence Metropolis-Hastings step that uses it on the
// RTT target P = |psi|^2 / Z (Sec. 3.3).
//
// Model: position d of the autoregressive order carries spin order[d]; input
// x_d = 1 - 2 s_order[d]; two ReLU hidden layers of width H; output logit_d,
// q(s_order[d] = 1 | s_<d) = sigmoid(logit_d).  Degrees: input d -> d+1,
// hidden unit k -> (k mod (N-1)) + 1, output d -> d+1; W1[k,d] kept iff
// m_k >= d+1, W2[k2,k1] iff m_k2 >= m_k1, W3[d,k] iff d+1 > m_k.
//
// Arithmetic (FP32 SIMT): every matrix product accumulates each output from
// its bias with one fma per term in increasing contraction index.  Ancestral
// sampling builds the first hidden layer incrementally in the same order, so
// the conditionals it samples from, and the log q it reports, are bit for
// bit those of the full forward pass: the acceptance test uses exactly the
// density the proposal was drawn from.
//
// Inference (sampling, log q for the acceptance test) can run its H x H layer
// on the tensor cores: h1 = ReLU(first layer) rounded to BF16, W2 (masked)
// in BF16, FP32 accumulation in tensor memory (tcgen05.mma kind::f16), bias
// and ReLU in the epilogue.  Sampling and evaluation run the same kernel on
// bit-identical BF16 inputs, so the density the proposal is drawn from is
// still exactly the one the acceptance test evaluates; training stays FP32.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>

#include "rtt_internal.cuh"
#include "rtt_tcgen05.cuh"

struct rtt_made_s {
    int device = 0, N = 0, H = 0;
    uint64_t seed = 0;
    int64_t P = 0;        // number of parameters
    int64_t step = 0;     // Adam step counter
    int32_t *d_order = nullptr;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
    float *d_mask = nullptr;   // masks of W1, W2, W3 in parameter layout (1 elsewhere)
    // workspace for batches of up to cap rows
    int64_t cap = 0;
    float *d_x = nullptr, *d_h1 = nullptr, *d_h2 = nullptr, *d_lg = nullptr;
    float *d_d3 = nullptr, *d_dh2 = nullptr, *d_dh1 = nullptr;
    double *d_logq = nullptr, *d_nll_parts = nullptr;
    uint8_t *d_prop = nullptr;          // proposals [cap][N]
    rtt_chain_state *d_pstate = nullptr;
    double *d_plogq = nullptr;
    uint8_t *d_batch = nullptr;         // gathered minibatch [batch_cap][N] (training loop)
    int64_t batch_cap = 0;
    double *d_fit = nullptr;            // per-epoch NLL sums + one batch NLL [fit_cap + 1]
    int32_t fit_cap = 0;
    size_t off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_W3 = 0, off_b3 = 0;
    // BF16 tensor-core inference of the H x H layer (when H allows it)
    int infer_bf16 = 0;
    int train_tc = 0;                  // training GEMMs on the tensor cores (BF16 hi/lo)
    __nv_bfloat16 *d_w2b = nullptr;    // [H][H] masked W2, row n = output unit, K-major
    __nv_bfloat16 *d_h1b = nullptr;    // [cap][H] ReLU(first layer) in BF16
    int *d_err = nullptr;              // bit 0: a bounded wait of the layer kernel expired
    CUtensorMap map_w2;
};

namespace mk {

constexpr uint64_t MADE_STREAM = 0x4D414445ull;

__device__ __forceinline__ double log_sigmoid(double y) {
    return fmin(y, 0.0) - log1p(exp(-fabs(y)));
}

// C[m][n] = epi(bias[n] + sum_k opA[m][k] opB[k][n]), fma in increasing k.
// opA[m][k] = TA ? A[k lda + m] : A[m lda + k];  opB[k][n] = TB ? B[n ldb + k] : B[k ldb + n]
// epi: ReLU (relu), * [gate[m][n] > 0] (gate), * mask[m][n] (mask); leading dim ldc.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float *__restrict__ A,
                                              int lda, const float *__restrict__ B, int ldb,
                                              float *__restrict__ C, int ldc,
                                              const float *__restrict__ bias, int relu,
                                              const float *__restrict__ gate,
                                              const float *__restrict__ mask) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            acc[i][j] = (bias && n < N) ? bias[n] : 0.f;
        }
    for (int k0 = 0; k0 < K; k0 += 16) {
        // 16 x 64 tiles, 4 elements per thread each
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + 256 * r;   // 0..1023
            const int kk = e >> 6, mm = e & 63;
            const int k = k0 + kk;
            const int m = m0 + mm, n = n0 + mm;
            float av = 0.f, bv = 0.f;
            if (k < K && m < M) av = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            if (k < K && n < N) bv = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            As[kk][mm] = av;
            Bs[kk][mm] = bv;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m >= M || n >= N) continue;
            float c = acc[i][j];
            if (relu) c = fmaxf(c, 0.f);
            if (gate && !(gate[(size_t)m * ldc + n] > 0.f)) c = 0.f;
            if (mask) c *= mask[(size_t)m * ldc + n];
            C[(size_t)m * ldc + n] = c;
        }
}

// inputs in autoregressive order: x[b][d] = 1 - 2 s[b][order[d]]
__global__ void k_inputs(const uint8_t *__restrict__ s, int64_t B, int N,
                         const int32_t *__restrict__ order, float *__restrict__ x) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * N) return;
    const int64_t b = t / N;
    const int d = (int)(t % N);
    x[t] = 1.f - 2.f * (float)s[b * N + order[d]];
}

// log q per row (double, increasing d) and, if d3, the NLL gradient
// (sigmoid(logit) - t) / B; nll_parts[b] = -log q
__global__ void k_loss(const float *__restrict__ lg, const uint8_t *__restrict__ s, int64_t B,
                       int N, const int32_t *__restrict__ order, double *__restrict__ logq,
                       float *__restrict__ d3) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double acc = 0.0;
    for (int d = 0; d < N; ++d) {
        const double y = (double)lg[b * N + d];
        const int t = s[b * N + order[d]];
        acc += log_sigmoid(t ? y : -y);
        if (d3) {
            const double sg = 1.0 / (1.0 + exp(-y));
            d3[b * N + d] = (float)((sg - (double)t) / (double)B);
        }
    }
    logq[b] = acc;
}

// The training loss: one warp per row b, lane l taking d = l, l + 32, ...;
// d3 as in k_loss (the same FP64 expression per entry), and log q(s_b) summed
// in the lanes' order then across the warp (only the minibatch NLL uses it).
__global__ void k_loss_train(const float *__restrict__ lg, const uint8_t *__restrict__ s, int64_t B,
                             int N, const int32_t *__restrict__ order, double *__restrict__ logq,
                             float *__restrict__ d3) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    double acc = 0.0;
    for (int d = lane; d < N; d += 32) {
        const double y = (double)lg[b * N + d];
        const int t = s[b * N + order[d]];
        acc += log_sigmoid(t ? y : -y);
        const double sg = 1.0 / (1.0 + exp(-y));
        d3[b * N + d] = (float)((sg - (double)t) / (double)B);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) logq[b] = acc;
}

// out[n] = sum_b D[b][n]: block (32 columns) x (32 row groups); thread (x, y)
// sums rows y, y + 32, ... of column x in increasing order, then the 32 partial
// sums of a column are added in increasing y
__global__ void __launch_bounds__(1024) k_colsum_par(const float *__restrict__ D, int64_t B, int N,
                                                     float *__restrict__ out) {
    __shared__ float part[32][33];
    const int x = threadIdx.x, y = threadIdx.y;
    const int n = blockIdx.x * 32 + x;
    float acc = 0.f;
    if (n < N)
        for (int64_t b = y; b < B; b += 32) acc += D[b * N + n];
    part[y][x] = acc;
    __syncthreads();
    if (y == 0 && n < N) {
        float t = 0.f;
        for (int i = 0; i < 32; ++i) t += part[i][x];
        out[n] = t;
    }
}

__global__ void k_sum_neg(const double *__restrict__ x, int64_t n, double *__restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += x[i];
    *out = -acc / (double)n;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    p[i] = p[i] - lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_fill_rows(float *__restrict__ x, int64_t B, int H, const float *__restrict__ b) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * H) return;
    x[t] = b[t % H];
}

__global__ void k_relu(const float *__restrict__ x, float *__restrict__ y, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    y[t] = fmaxf(x[t], 0.f);
}

// Position d of ancestral sampling, one thread per chain: logit_d from h2
// (bias then increasing k, as the forward product), draw the bit, add its
// log-probability, then add input d into the first-layer pre-activations.
__global__ void k_sample_pos(int d, int64_t B, int N, int H, const float *__restrict__ W1,
                             const float *__restrict__ W3, const float *__restrict__ b3,
                             const float *__restrict__ h2, float *__restrict__ h1pre,
                             const int32_t *__restrict__ order, uint8_t *__restrict__ spins,
                             double *__restrict__ logq, uint64_t seed, int64_t chain0,
                             int64_t round) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float lg = b3[d];
    const float *w = W3 + (size_t)d * H;
    const float *hb = h2 + (size_t)b * H;
    for (int k = 0; k < H; ++k) lg = fmaf(hb[k], w[k], lg);
    const double y = (double)lg;
    uint64_t r[4];
    rttd::philox4x64_10((uint64_t)(chain0 + b), (uint64_t)round, (uint64_t)d, 0ull, seed,
                        MADE_STREAM, r);
    const double u = (double)(r[0] >> 11) * 0x1.0p-53;
    const double pr = 1.0 / (1.0 + exp(-y));
    const int t = u < pr ? 1 : 0;
    logq[b] = (d == 0 ? 0.0 : logq[b]) + log_sigmoid(t ? y : -y);
    spins[b * N + order[d]] = (uint8_t)t;
    const float x = t ? -1.f : 1.f;
    float *h = h1pre + (size_t)b * H;
    for (int k = 0; k < H; ++k) h[k] = fmaf(x, W1[(size_t)k * N + d], h[k]);
}

// Independence Metropolis-Hastings decision, one thread per chain.
__global__ void k_indep_decide(int64_t B, int N, uint8_t *__restrict__ spins,
                               rtt_chain_state *__restrict__ state, const double *__restrict__ logq,
                               const uint8_t *__restrict__ prop,
                               const rtt_chain_state *__restrict__ pstate,
                               const double *__restrict__ plogq, uint64_t seed, int64_t chain0,
                               int64_t round, int64_t *__restrict__ n_accept) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double m0 = state[b].mant, m1 = pstate[b].mant;
    const double la0 = (m0 == 0.0) ? -INFINITY : (double)state[b].exp2 * 0.6931471805599453 + log(fabs(m0));
    const double la1 = (m1 == 0.0) ? -INFINITY : (double)pstate[b].exp2 * 0.6931471805599453 + log(fabs(m1));
    uint64_t r[4];
    rttd::philox4x64_10((uint64_t)(chain0 + b), (uint64_t)round, (uint64_t)N, 0ull, seed, MADE_STREAM, r);
    const double u = (double)(r[0] >> 11) * 0x1.0p-53;
    const double lhs = log(u);
    const double rhs = 2.0 * (la1 - la0) + logq[b] - plogq[b];
    const bool accept = (m1 != 0.0) && isfinite(m1) && (u == 0.0 || lhs < rhs);
    if (!accept) return;
    for (int i = 0; i < N; ++i) spins[b * N + i] = prop[b * N + i];
    state[b] = pstate[b];
    if (n_accept) n_accept[b] += 1;
}

// BF16 (round to nearest) of ReLU(x), and of the masked second-layer weights
__global__ void k_relu_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(fmaxf(x[i], 0.f));
}
__global__ void k_w2_bf16(const float *__restrict__ w, const float *__restrict__ mask,
                          __nv_bfloat16 *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(w[i] * mask[i]);
}

// h2[m][n] = ReLU(b2[n] + sum_k h1[m][k] W2[n][k]) for one 128-row tile and all
// H columns: A (h1, 128 x 64 per K chunk) and B (W2, H x 64 per chunk) by TMA
// into a two-stage ring (128-byte swizzle, K-major), thread 0 issues the MMAs
// (M = 128, N = min(H, 256), K = 16 each) into an H-column FP32 accumulator in
// tensor memory; the epilogue (thread = row = TMEM lane) adds the bias, applies
// ReLU and stores the row.  Every wait is bounded: on expiry the CTA sets bit 0
// of err, drains its own copies, frees its tensor memory and returns.
constexpr int L2_THREADS = 128;
__global__ void __launch_bounds__(L2_THREADS, 1)
    k_l2_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
            const float *__restrict__ bias, float *__restrict__ out, int64_t B, int H, int tcols,
            const float *__restrict__ w3row, const float *__restrict__ b3d, float *__restrict__ lg_out,
            int *__restrict__ err, long long wait_limit) {
    using namespace tcd;
    extern __shared__ __align__(1024) uint8_t l2_smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (sa(l2_smem) + 1023u) & ~1023u;
    const uint32_t A_BYTES = 128u * 128u, B_BYTES = (uint32_t)H * 128u, STAGE = A_BYTES + B_BYTES;
    const uint32_t ctrl = base + 2u * STAGE;
    auto full_bar = [&](int st) { return ctrl + 8u * (uint32_t)st; };
    auto empty_bar = [&](int st) { return ctrl + 16u + 8u * (uint32_t)st; };
    const uint32_t done_bar = ctrl + 32u;
    uint32_t *tmem_slot = (uint32_t *)(l2_smem + (ctrl + 40u - sa(l2_smem)));
    volatile int *abort_flag = (volatile int *)(l2_smem + (ctrl + 44u - sa(l2_smem)));
    const int64_t m0 = (int64_t)blockIdx.x * 128;
    const int nmma = H > 256 ? 256 : H;           // N of one MMA
    const int nsub = H / nmma;
    const int brows = H > 256 ? 256 : H;          // rows of one B box
    const int nbox = H / brows;
    const int nK = H / 64;
    const uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nmma >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            mbar_init(full_bar(st), 1);
            mbar_init(empty_bar(st), 1);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(sa(tmem_slot), (uint32_t)tcols);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0, waited = 0;
    auto issue = [&](int c) {
        const int st = c & 1;
        const uint32_t a_dst = base + (uint32_t)st * STAGE, b_dst = a_dst + A_BYTES;
        mbar_expect_tx(full_bar(st), STAGE);
        tma_load_2d(a_dst, &map_a, c * 64, (int)m0, full_bar(st));
        for (int r = 0; r < nbox; ++r)
            tma_load_2d(b_dst + (uint32_t)r * (uint32_t)brows * 128u, &map_b, c * 64, r * brows,
                        full_bar(st));
        ++issued;
    };
    if (tid == 0) {
        issue(0);
        if (nK > 1) issue(1);
        for (int c = 0; c < nK; ++c) {
            const int st = c & 1;
            if (!mbar_wait(full_bar(st), (uint32_t)((c >> 1) & 1), wait_limit)) {
                atomicOr(err, 1);
                *abort_flag = 1;
                break;
            }
            waited = c + 1;
            tc_after();
            const uint32_t a_src = base + (uint32_t)st * STAGE, b_src = a_src + A_BYTES;
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                const uint64_t adesc = sdesc(a_src + (uint32_t)kb * 32u);
                for (int ns = 0; ns < nsub; ++ns) {
                    const uint64_t bdesc = sdesc(b_src + (uint32_t)ns * (uint32_t)nmma * 128u +
                                                 (uint32_t)kb * 32u);
                    mma_bf16(tmem + (uint32_t)(ns * nmma), adesc, bdesc, IDESC,
                             (c | kb) != 0 ? 1u : 0u);
                }
            }
            mma_commit(empty_bar(st));
            if (c + 2 < nK) {
                if (!mbar_wait(empty_bar(st), (uint32_t)((c >> 1) & 1), wait_limit)) {
                    atomicOr(err, 1);
                    *abort_flag = 1;
                    break;
                }
                issue(c + 2);
            }
        }
        mma_commit(done_bar);       // arrives once every MMA issued so far is done
    }
    if (!mbar_wait(done_bar, 0u, wait_limit)) {
        atomicOr(err, 1);
        *abort_flag = 1;
    }
    tc_after();
    __syncthreads();
    if (!*abort_flag) {
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
        float *orow = out ? out + (row < B ? row : 0) * (int64_t)H : nullptr;
        float lg = lg_out ? *b3d : 0.f;  // logit mode: b3[d] + sum_n h2[n] W3[d][n], increasing n
        for (int c0 = 0; c0 < H; c0 += 64) {
            uint32_t x[32], y[32];
            tmem_ld_2x32(tw + (uint32_t)c0, tw + (uint32_t)c0 + 32u, x, y);
            if (lg_out) {
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    lg = fmaf(fmaxf(__uint_as_float(x[q]) + bias[c0 + q], 0.f), w3row[c0 + q], lg);
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    lg = fmaf(fmaxf(__uint_as_float(y[q]) + bias[c0 + 32 + q], 0.f), w3row[c0 + 32 + q],
                              lg);
            } else if (row < B) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float4 v;
                    v.x = fmaxf(__uint_as_float(x[4 * q + 0]) + bias[c0 + 4 * q + 0], 0.f);
                    v.y = fmaxf(__uint_as_float(x[4 * q + 1]) + bias[c0 + 4 * q + 1], 0.f);
                    v.z = fmaxf(__uint_as_float(x[4 * q + 2]) + bias[c0 + 4 * q + 2], 0.f);
                    v.w = fmaxf(__uint_as_float(x[4 * q + 3]) + bias[c0 + 4 * q + 3], 0.f);
                    *reinterpret_cast<float4 *>(orow + c0 + 4 * q) = v;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float4 v;
                    v.x = fmaxf(__uint_as_float(y[4 * q + 0]) + bias[c0 + 32 + 4 * q + 0], 0.f);
                    v.y = fmaxf(__uint_as_float(y[4 * q + 1]) + bias[c0 + 32 + 4 * q + 1], 0.f);
                    v.z = fmaxf(__uint_as_float(y[4 * q + 2]) + bias[c0 + 32 + 4 * q + 2], 0.f);
                    v.w = fmaxf(__uint_as_float(y[4 * q + 3]) + bias[c0 + 32 + 4 * q + 3], 0.f);
                    *reinterpret_cast<float4 *>(orow + c0 + 32 + 4 * q) = v;
                }
            }
        }
        if (lg_out && row < B) lg_out[row] = lg;
    } else if (tid == 0) {
        // drain this CTA's own copies before the shared memory goes away
        for (int c = waited; c < issued; ++c)
            mbar_wait(full_bar(c & 1), (uint32_t)((c >> 1) & 1), wait_limit);
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)tcols);
}

// Feature-major forms for BF16 sampling ([H][B], thread = chain, so that a
// warp touches consecutive chains of one feature): the same arithmetic per
// element as the row-major kernels above.
__global__ void k_fill_T(float *__restrict__ xT, int64_t B, int H, const float *__restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * H) xT[i] = b[i / B];
}
// y[b][k] = bf16(ReLU(xT[k][b])) through a 32 x 32 shared-memory tile
__global__ void k_relu_bf16_T(const float *__restrict__ xT, __nv_bfloat16 *__restrict__ y,
                              int64_t B, int H) {
    __shared__ float t[32][33];
    const int64_t b0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r;
        const int64_t b = b0 + threadIdx.x;
        t[r][threadIdx.x] = (k < H && b < B) ? xT[(int64_t)k * B + b] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t b = b0 + r;
        const int k = k0 + threadIdx.x;
        if (b < B && k < H) y[b * H + k] = __float2bfloat16_rn(fmaxf(t[threadIdx.x][r], 0.f));
    }
}
// Position d of BF16 sampling, one thread per chain: the logit comes from the
// layer kernel's epilogue (bias, then increasing n, as the output product);
// draw the bit, add its log-probability, keep x_d = 1 - 2 s for the update.
__global__ void k_sample_bit(int d, int64_t B, int N, const float *__restrict__ lg,
                             const int32_t *__restrict__ order, uint8_t *__restrict__ spins,
                             double *__restrict__ logq, float *__restrict__ xs, uint64_t seed,
                             int64_t chain0, int64_t round) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double y = (double)lg[b];
    uint64_t r[4];
    rttd::philox4x64_10((uint64_t)(chain0 + b), (uint64_t)round, (uint64_t)d, 0ull, seed,
                        MADE_STREAM, r);
    const double u = (double)(r[0] >> 11) * 0x1.0p-53;
    const double pr = 1.0 / (1.0 + exp(-y));
    const int t = u < pr ? 1 : 0;
    logq[b] = (d == 0 ? 0.0 : logq[b]) + log_sigmoid(t ? y : -y);
    spins[b * N + order[d]] = (uint8_t)t;
    xs[b] = t ? -1.f : 1.f;
}
// add input d to the feature-major pre-activations, h1preT[k][b] += x_b W1[k][d]
// (the forward product's next fma), and write bf16(ReLU) of the result to the
// row-major h1b[b][k] through a 32 x 32 shared-memory tile
__global__ void k_h1_update_bf16_T(int d, int64_t B, int N, int H, const float *__restrict__ W1,
                                   const float *__restrict__ xs, float *__restrict__ h1preT,
                                   __nv_bfloat16 *__restrict__ y) {
    __shared__ float t[32][33];
    const int64_t b0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r;
        const int64_t b = b0 + threadIdx.x;
        float v = 0.f;
        if (k < H && b < B) {
            float *h = h1preT + (int64_t)k * B + b;
            v = fmaf(xs[b], W1[(size_t)k * N + d], *h);
            *h = v;
        }
        t[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t b = b0 + r;
        const int k = k0 + threadIdx.x;
        if (b < B && k < H) y[b * H + k] = __float2bfloat16_rn(fmaxf(t[threadIdx.x][r], 0.f));
    }
}

// masks in parameter layout (1 on biases)
__global__ void k_masks(float *__restrict__ mask, int N, int H, size_t oW1, size_t oW2, size_t oW3,
                        int64_t P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    auto deg = [&](int k) { return N > 1 ? (k % (N - 1)) + 1 : 1; };
    float v = 1.f;
    if (i >= (int64_t)oW1 && i < (int64_t)(oW1 + (size_t)H * N)) {
        const int64_t e = i - oW1;
        const int k = (int)(e / N), d = (int)(e % N);
        v = deg(k) >= d + 1 ? 1.f : 0.f;
    } else if (i >= (int64_t)oW2 && i < (int64_t)(oW2 + (size_t)H * H)) {
        const int64_t e = i - oW2;
        const int k2 = (int)(e / H), k1 = (int)(e % H);
        v = deg(k2) >= deg(k1) ? 1.f : 0.f;
    } else if (i >= (int64_t)oW3 && i < (int64_t)(oW3 + (size_t)N * H)) {
        const int64_t e = i - oW3;
        const int d = (int)(e / H), k = (int)(e % H);
        v = (d + 1) > deg(k) ? 1.f : 0.f;
    }
    mask[i] = v;
}

__global__ void k_mul(float *__restrict__ x, const float *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= y[i];
}

// Minibatch shuffle of the training loop: a keyed permutation of [0, n)
// per epoch, computed row by row with no sort.  A balanced Feistel network
// (four rounds, each half of 2h bits mixed by the 64-bit finaliser of
// MurmurHash3 keyed by seed, epoch and round) permutes [0, 4^h) with
// 4^h >= n; values at or beyond n walk the permutation's cycle until they
// land inside [0, n) (Black and Rogaway, "Ciphers with arbitrary finite
// domains", 2002), which restricts it to a permutation of [0, n).
struct Shuffle {
    uint64_t n = 1, key = 0;
    int h = 0;
    uint64_t mask = 0;
};
__host__ __device__ inline uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}
__host__ __device__ inline Shuffle shuffle_of(uint64_t n, uint64_t seed, int64_t epoch) {
    Shuffle s;
    s.n = n > 0 ? n : 1;
    s.key = fmix64(seed ^ fmix64((uint64_t)epoch + 0x9e3779b97f4a7c15ull));
    int h = 1;
    while (h < 31 && ((uint64_t)1 << (2 * h)) < s.n) ++h;
    s.h = h;
    s.mask = ((uint64_t)1 << h) - 1;
    return s;
}
__host__ __device__ inline uint64_t feistel(const Shuffle &s, uint64_t x) {
    uint64_t l = x >> s.h, r = x & s.mask;
    for (int k = 0; k < 4; ++k) {
        const uint64_t f = fmix64(r ^ (s.key + 0x632be59bd9b4e019ull * (uint64_t)(k + 1))) & s.mask;
        const uint64_t t = l ^ f;
        l = r;
        r = t;
    }
    return (l << s.h) | r;
}
// image of i < n; the walk ends because the cycle through i holds i itself
__host__ __device__ inline uint64_t shuffle_index(const Shuffle &s, uint64_t i) {
    uint64_t x = feistel(s, i);
    while (x >= s.n) x = feistel(s, x);
    return x;
}

// out[r][:] = data[shuffle(first + r)][:], r < rows (one block per row)
__global__ void k_gather_rows(const uint8_t *__restrict__ data, Shuffle sh, int64_t first,
                              int64_t rows, int N, uint8_t *__restrict__ out) {
    const int64_t r = blockIdx.x;
    if (r >= rows) return;
    const uint64_t src = shuffle_index(sh, (uint64_t)(first + r));
    for (int i = threadIdx.x; i < N; i += blockDim.x) out[r * N + i] = data[src * N + i];
}

// acc[e] += x (one thread)
__global__ void k_accumulate(double *__restrict__ acc, const double *__restrict__ x) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *acc += *x;
}

// ---------------------------------------------------------------- tensor-core training GEMM
// The same C = epi(bias + opA . opB) as k_gemm on the 5th-generation tensor
// cores, for training: each FP32 operand is split into BF16 hi + lo (x = hi +
// lo + O(2^-18 |x|)), and three products hi.hi + hi.lo + lo.hi accumulate in
// FP32 in tensor memory (the dropped lo.lo is O(2^-18) too).  One 128 x 128
// tile of C per CTA of 128 threads (thread = row of the tile in the
// epilogue); K in blocks of 64: all threads read a block of both operands in
// FP32 (either orientation, zero past the edges), split it and store it into
// a two-stage shared-memory ring in the 128-byte-swizzled K-major layout;
// thread 0 issues the block's 12 MMAs (M = N = 128, K = 16) and commits them
// to the stage's mbarrier, which the threads wait on before they refill the
// stage.  Every wait is bounded; on expiry the CTA records bit 0 in err,
// skips the rest and writes nothing.
constexpr int GT_THREADS = 128;
constexpr uint32_t GT_TILE = 128u * 128u;              // bytes of one 128 x 64 BF16 tile
constexpr uint32_t GT_STAGE = 4u * GT_TILE;            // A hi, A lo, B hi, B lo
constexpr uint32_t GT_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);  // BF16 x BF16 -> FP32, K-major, 128 x 128
constexpr size_t GT_SMEM = 1024 + 2 * (size_t)GT_STAGE + 64;

__device__ __forceinline__ void gt_split8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * p], v[2 * p + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * p] - hf.x, v[2 * p + 1] - hf.y);
        h[p] = *reinterpret_cast<const uint32_t *>(&hb);
        l[p] = *reinterpret_cast<const uint32_t *>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ void gt_st16(uint32_t addr, const uint4 &v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(GT_THREADS, 1)
    k_gemm_tc(int M, int N, int K, const float *__restrict__ A, int lda, const float *__restrict__ B,
              int ldb, float *__restrict__ C, int ldc, const float *__restrict__ bias, int relu,
              const float *__restrict__ gate, const float *__restrict__ mask, int *err,
              long long limit) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t ring = tcd::sa(base);
    uint64_t *bars = (uint64_t *)(base + 2 * GT_STAGE);
    const uint32_t bar0 = tcd::sa(bars);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
    if (warp == 0) tcd::tmem_alloc(tcd::sa(tmem_slot), 128u);
    if (tid == 0) {
        tcd::mbar_init(bar0, 1);
        tcd::mbar_init(bar0 + 8u, 1);
        *abort_flag = 0;
        tcd::fence_barrier_init();
    }
    tcd::tc_before();
    __syncthreads();
    tcd::tc_after();
    const uint32_t tmem = *tmem_slot;
    const int nkb = (K + 63) / 64;
    // element (r, k) of a 128 x 64 operand tile: opA[m0 + r][k] or opB[k][n0 + r]
    auto elem_a = [&](int r, int k) -> float {
        const int m = m0 + r;
        if (m >= M || k >= K) return 0.f;
        return TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
    };
    auto elem_b = [&](int r, int k) -> float {
        const int n = n0 + r;
        if (n >= N || k >= K) return 0.f;
        return TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
    };
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb & 1;
        if (kb >= 2 && !*abort_flag) {
            // the MMAs of block kb - 2 have read this stage
            if (!tcd::mbar_wait(bar0 + 8u * s, (uint32_t)(((kb - 2) >> 1) & 1), limit)) {
                atomicOr(err, 1);
                *abort_flag = 1;
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        const uint32_t st = ring + (uint32_t)s * GT_STAGE;
        // thread tid fills row tid of the four tiles, 8 K-entries at a time
        const int k0 = kb * 64;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float va[8], vb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                va[i] = elem_a(tid, k0 + 8 * c + i);
                vb[i] = elem_b(tid, k0 + 8 * c + i);
            }
            uint4 ah, al, bh, bl;
            gt_split8(va, ah, al);
            gt_split8(vb, bh, bl);
            const uint32_t off = (uint32_t)tid * 128u + ((uint32_t)(c ^ (tid & 7)) << 4);
            gt_st16(st + off, ah);
            gt_st16(st + GT_TILE + off, al);
            gt_st16(st + 2 * GT_TILE + off, bh);
            gt_st16(st + 3 * GT_TILE + off, bl);
        }
        tcd::fence_async_smem();
        tcd::tc_before();
        __syncthreads();
        if (tid == 0) {
            tcd::tc_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t o = (uint32_t)(kk * 32);
                const uint64_t ah = tcd::sdesc(st + o), al = tcd::sdesc(st + GT_TILE + o);
                const uint64_t bh = tcd::sdesc(st + 2 * GT_TILE + o), bl = tcd::sdesc(st + 3 * GT_TILE + o);
                tcd::mma_bf16(tmem, ah, bh, GT_IDESC, (kb | kk) ? 1u : 0u);
                tcd::mma_bf16(tmem, ah, bl, GT_IDESC, 1u);
                tcd::mma_bf16(tmem, al, bh, GT_IDESC, 1u);
            }
            tcd::mma_commit(bar0 + 8u * s);
        }
    }
    // the last block's MMAs complete after every earlier one
    if (nkb > 0 && !*abort_flag) {
        const int kl = nkb - 1;
        if (!tcd::mbar_wait(bar0 + 8u * (kl & 1), (uint32_t)((kl >> 1) & 1), limit)) {
            atomicOr(err, 1);
            *abort_flag = 1;
        }
    }
    tcd::tc_after();
    __syncthreads();
    if (!*abort_flag) {
        const int m = m0 + tid;
        const uint32_t tq = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int cb = 0; cb < 128; cb += 64) {
            uint32_t x0[32], x1[32];
            if (nkb > 0) {
                tcd::tmem_ld_2x32(tq + (uint32_t)cb, tq + (uint32_t)cb + 32u, x0, x1);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) x0[i] = x1[i] = 0u;
            }
            if (m < M) {
#pragma unroll
                for (int i = 0; i < 64; ++i) {
                    const int n = n0 + cb + i;
                    if (n < N) {
                        float c = __uint_as_float(i < 32 ? x0[i] : x1[i - 32]);
                        if (bias) c += bias[n];
                        if (relu) c = fmaxf(c, 0.f);
                        if (gate && !(gate[(size_t)m * ldc + n] > 0.f)) c = 0.f;
                        if (mask) c *= mask[(size_t)m * ldc + n];
                        C[(size_t)m * ldc + n] = c;
                    }
                }
            }
        }
    }
    tcd::tc_before();
    __syncthreads();
    tcd::tc_after();
    if (warp == 0) tcd::tmem_dealloc(tmem, 128u);
}

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
                 int ldc, const float *bias, int relu, const float *gate, const float *mask,
                 cudaStream_t st) {
    dim3 grid(nb(N, 64), nb(M, 64));
    k_gemm<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, gate, mask);
    return cudaGetLastError();
}
// the training GEMM: tensor cores (BF16 hi/lo, three products) or k_gemm
template <bool TA, bool TB>
cudaError_t gemm_train(bool tc, int *err, int M, int N, int K, const float *A, int lda,
                       const float *B, int ldb, float *C, int ldc, const float *bias, int relu,
                       const float *gate, const float *mask, cudaStream_t st) {
    if (!tc) return gemm<TA, TB>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, gate, mask, st);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GT_SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid(nb(N, 128), nb(M, 128));
    k_gemm_tc<TA, TB><<<grid, GT_THREADS, GT_SMEM, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu,
                                                          gate, mask, err, 4000000000LL);
    return cudaGetLastError();
}

}  // namespace mk

// ============================================================================ host
namespace {

rtt_status mfail(rtt_status s, const std::string &m) {
    rtt_set_error(m);
    return s;
}
rtt_status mcuda(cudaError_t e, const char *w) {
    return mfail(e == cudaErrorMemoryAllocation ? RTT_ERR_OOM : RTT_ERR_CUDA,
                 std::string(w) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define MC(expr, w)                                                                                \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return mcuda(_e, w);                                                \
    } while (0)

struct MGuard {
    int prev = -1;
    bool changed = false;
    explicit MGuard(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) changed = cudaSetDevice(d) == cudaSuccess;
    }
    ~MGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

void free_ws(rtt_made_s *m) {
    void *bufs[] = {m->d_x, m->d_h1, m->d_h2, m->d_lg, m->d_d3, m->d_dh2, m->d_dh1,
                    m->d_logq, m->d_nll_parts, m->d_prop, m->d_pstate, m->d_plogq, m->d_h1b};
    for (void *b : bufs) cudaFree(b);
    m->d_x = m->d_h1 = m->d_h2 = m->d_lg = m->d_d3 = m->d_dh2 = m->d_dh1 = nullptr;
    m->d_logq = m->d_nll_parts = m->d_plogq = nullptr;
    m->d_prop = nullptr;
    m->d_pstate = nullptr;
    m->d_h1b = nullptr;
    m->cap = 0;
}

rtt_status ensure_ws(rtt_made_s *m, int64_t B) {
    if (B <= m->cap) return RTT_OK;
    MC(cudaDeviceSynchronize(), "made workspace");
    free_ws(m);
    const size_t N = m->N, H = m->H;
    MC(cudaMalloc((void **)&m->d_x, B * N * 4), "made ws");
    MC(cudaMalloc((void **)&m->d_h1, B * H * 4), "made ws");
    MC(cudaMalloc((void **)&m->d_h2, B * H * 4), "made ws");
    MC(cudaMalloc((void **)&m->d_h1b, B * H * 2), "made ws");
    MC(cudaMalloc((void **)&m->d_lg, B * N * 4), "made ws");
    MC(cudaMalloc((void **)&m->d_d3, B * N * 4), "made ws");
    MC(cudaMalloc((void **)&m->d_dh2, B * H * 4), "made ws");
    MC(cudaMalloc((void **)&m->d_dh1, B * H * 4), "made ws");
    MC(cudaMalloc((void **)&m->d_logq, B * 8), "made ws");
    MC(cudaMalloc((void **)&m->d_nll_parts, B * 8), "made ws");
    MC(cudaMalloc((void **)&m->d_prop, B * N), "made ws");
    MC(cudaMalloc((void **)&m->d_pstate, B * sizeof(rtt_chain_state)), "made ws");
    MC(cudaMalloc((void **)&m->d_plogq, B * 8), "made ws");
    m->cap = B;
    return RTT_OK;
}

// forward pass for rows of spins -> m->d_h1, d_h2, d_lg (and x)
// (train: the training GEMMs, tensor cores when m->train_tc; else FP32 k_gemm)
rtt_status forward(rtt_made_s *m, const uint8_t *spins, int64_t B, cudaStream_t st, bool train = false) {
    const int N = m->N, H = m->H;
    const float *p = m->d_p;
    const bool tc = train && m->train_tc;
    mk::k_inputs<<<mk::nb(B * N, 256), 256, 0, st>>>(spins, B, N, m->d_order, m->d_x);
    MC(cudaGetLastError(), "made inputs");
    MC((mk::gemm_train<false, true>(tc, m->d_err, (int)B, H, N, m->d_x, N, p + m->off_W1, N, m->d_h1,
                                    H, p + m->off_b1, 1, nullptr, nullptr, st)), "made layer 1");
    MC((mk::gemm_train<false, true>(tc, m->d_err, (int)B, H, H, m->d_h1, H, p + m->off_W2, H, m->d_h2,
                                    H, p + m->off_b2, 1, nullptr, nullptr, st)), "made layer 2");
    MC((mk::gemm_train<false, true>(tc, m->d_err, (int)B, N, H, m->d_h2, H, p + m->off_W3, H, m->d_lg,
                                    N, p + m->off_b3, 0, nullptr, nullptr, st)), "made output");
    return RTT_OK;
}

// H values the tensor-core layer takes: multiples of 64 up to 512 that are
// one or two MMA widths (N <= 256)
bool l2_tc_supported(int H) {
    if (H < 64 || H > 512 || H % 64) return false;
    const int nmma = H > 256 ? 256 : H;
    return H % nmma == 0;
}
int l2_tcols(int H) {
    int c = 32;
    while (c < H) c <<= 1;
    return c;
}
size_t l2_smem(int H) {
    const size_t stage = (size_t)128 * 128 + (size_t)H * 128;
    // at least 164 KB, so that no other tensor-memory kernel shares the SM
    return std::max((size_t)1024 + 2 * stage + 64, (size_t)164 * 1024);
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// row-major bf16 matrix [rows][cols] (cols = K, a multiple of 64), boxes of
// 64 K-elements x box_rows rows, 128-byte swizzle, rows past the end read as 0
bool encode_bf16(CUtensorMap *map, const void *ptr, int64_t rows, int cols, int box_rows) {
    EncodeTiled enc = (EncodeTiled)tc_encode_tiled_fn();
    if (!enc) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estride[2] = {1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), gdim, gstride, box,
               estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the masked W2 in BF16 (before every inference call: parameters may have changed)
rtt_status refresh_w2(rtt_made_s *m, cudaStream_t st) {
    const int64_t n = (int64_t)m->H * m->H;
    mk::k_w2_bf16<<<mk::nb(n, 256), 256, 0, st>>>(m->d_p + m->off_W2, m->d_mask + m->off_W2,
                                                   m->d_w2b, n);
    MC(cudaGetLastError(), "made W2 to BF16");
    return RTT_OK;
}

// h2 = ReLU(b2 + h1b W2b^T) on the tensor cores, h1b already filled; with
// d >= 0 only the logit of position d per row goes to m->d_lg (h2 is not stored)
rtt_status layer2_tc(rtt_made_s *m, int64_t B, cudaStream_t st, int d = -1) {
    const int H = m->H;
    CUtensorMap map_a;
    if (!encode_bf16(&map_a, m->d_h1b, B, H, 128))
        return mfail(RTT_ERR_CUDA, "made layer 2: cuTensorMapEncodeTiled failed");
    const size_t smem = l2_smem(H);
    MC(cudaFuncSetAttribute(mk::k_l2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
       "made layer 2 attributes");
    mk::k_l2_tc<<<(unsigned)((B + 127) / 128), mk::L2_THREADS, smem, st>>>(
        map_a, m->map_w2, m->d_p + m->off_b2, d >= 0 ? nullptr : m->d_h2, B, H, l2_tcols(H),
        d >= 0 ? m->d_p + m->off_W3 + (size_t)d * H : nullptr,
        d >= 0 ? m->d_p + m->off_b3 + d : nullptr,
        d >= 0 ? m->d_lg : nullptr, m->d_err, 4000000000LL);
    MC(cudaGetLastError(), "made layer 2 (tensor cores)");
    return RTT_OK;
}

// the inference forward pass: as forward(), with the H x H layer on the
// tensor cores when inference runs in BF16
rtt_status forward_infer(rtt_made_s *m, const uint8_t *spins, int64_t B, cudaStream_t st) {
    if (!m->infer_bf16) return forward(m, spins, B, st);
    const int N = m->N, H = m->H;
    const float *p = m->d_p;
    mk::k_inputs<<<mk::nb(B * N, 256), 256, 0, st>>>(spins, B, N, m->d_order, m->d_x);
    MC(cudaGetLastError(), "made inputs");
    MC((mk::gemm<false, true>((int)B, H, N, m->d_x, N, p + m->off_W1, N, m->d_h1, H,
                              p + m->off_b1, 1, nullptr, nullptr, st)), "made layer 1");
    mk::k_relu_bf16<<<mk::nb(B * H, 256), 256, 0, st>>>(m->d_h1, m->d_h1b, B * H);
    MC(cudaGetLastError(), "made layer 1 to BF16");
    rtt_status s = layer2_tc(m, B, st);
    if (s != RTT_OK) return s;
    MC((mk::gemm<false, true>((int)B, N, H, m->d_h2, H, p + m->off_W3, H, m->d_lg, N,
                              p + m->off_b3, 0, nullptr, nullptr, st)), "made output");
    return RTT_OK;
}

// gradient of the mean NLL into m->d_g (masked); nll into *nll_dev if given
rtt_status gradients(rtt_made_s *m, const uint8_t *spins, int64_t B, double *nll_dev,
                     cudaStream_t st) {
    const int N = m->N, H = m->H;
    const float *p = m->d_p;
    float *g = m->d_g;
    rtt_status s = forward(m, spins, B, st, true);
    const bool tc = m->train_tc != 0;
    if (s != RTT_OK) return s;
    mk::k_loss_train<<<mk::nb(B * 32, 256), 256, 0, st>>>(m->d_lg, spins, B, N, m->d_order, m->d_logq,
                                                          m->d_d3);
    MC(cudaGetLastError(), "made loss");
    if (nll_dev) {
        mk::k_sum_neg<<<1, 1, 0, st>>>(m->d_logq, B, nll_dev);
        MC(cudaGetLastError(), "made nll");
    }
    const float *mask = m->d_mask;
    // output layer: dW3 = d3^T h2 (masked), db3 = colsum d3
    MC((mk::gemm_train<true, false>(tc, m->d_err, N, H, (int)B, m->d_d3, N, m->d_h2, H, g + m->off_W3, H, nullptr, 0,
                              nullptr, mask + m->off_W3, st)), "made dW3");
    mk::k_colsum_par<<<mk::nb(N, 32), dim3(32, 32), 0, st>>>(m->d_d3, B, N, g + m->off_b3);
    // dh2 = (d3 W3) * [h2 > 0]
    MC((mk::gemm_train<false, false>(tc, m->d_err, (int)B, H, N, m->d_d3, N, p + m->off_W3, H, m->d_dh2, H, nullptr, 0,
                               m->d_h2, nullptr, st)), "made dh2");
    MC((mk::gemm_train<true, false>(tc, m->d_err, H, H, (int)B, m->d_dh2, H, m->d_h1, H, g + m->off_W2, H, nullptr, 0,
                              nullptr, mask + m->off_W2, st)), "made dW2");
    mk::k_colsum_par<<<mk::nb(H, 32), dim3(32, 32), 0, st>>>(m->d_dh2, B, H, g + m->off_b2);
    // dh1 = (dh2 W2) * [h1 > 0]
    MC((mk::gemm_train<false, false>(tc, m->d_err, (int)B, H, H, m->d_dh2, H, p + m->off_W2, H, m->d_dh1, H, nullptr, 0,
                               m->d_h1, nullptr, st)), "made dh1");
    MC((mk::gemm_train<true, false>(tc, m->d_err, H, N, (int)B, m->d_dh1, H, m->d_x, N, g + m->off_W1, N, nullptr, 0,
                              nullptr, mask + m->off_W1, st)), "made dW1");
    mk::k_colsum_par<<<mk::nb(H, 32), dim3(32, 32), 0, st>>>(m->d_dh1, B, H, g + m->off_b1);
    MC(cudaGetLastError(), "made gradients");
    return RTT_OK;
}

}  // namespace

extern "C" {

rtt_status rtt_made_create(int32_t n_spins, int32_t hidden, const int32_t *order,
                           const double *init_weights, uint64_t seed, int32_t device,
                           rtt_made *out) {
    if (!out || !order || !init_weights || n_spins < 1 || hidden < 1)
        return mfail(RTT_ERR_INVALID_ARG, "rtt_made_create: bad arguments");
    *out = nullptr;
    std::vector<int> seen(n_spins, 0);
    for (int d = 0; d < n_spins; ++d) {
        if (order[d] < 0 || order[d] >= n_spins || seen[order[d]]++)
            return mfail(RTT_ERR_INVALID_ARG, "rtt_made_create: order is not a permutation");
    }
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess)
        return mfail(RTT_ERR_CUDA, "rtt_made_create: cudaGetDevice");
    MGuard guard(dev);
    rtt_made_s *m = new rtt_made_s();
    m->device = dev;
    m->N = n_spins;
    m->H = hidden;
    m->seed = seed;
    const size_t N = n_spins, H = hidden;
    m->off_W1 = 0;
    m->off_b1 = H * N;
    m->off_W2 = m->off_b1 + H;
    m->off_b2 = m->off_W2 + H * H;
    m->off_W3 = m->off_b2 + H;
    m->off_b3 = m->off_W3 + N * H;
    m->P = (int64_t)(m->off_b3 + N);
    std::vector<float> hp(m->P);
    for (int64_t i = 0; i < m->P; ++i) hp[i] = (float)init_weights[i];
    auto cleanup = [&](rtt_status s) {
        rtt_made_destroy(m);
        return s;
    };
    cudaError_t e;
    if ((e = cudaMalloc((void **)&m->d_order, N * 4)) != cudaSuccess) return cleanup(mcuda(e, "made"));
    cudaMemcpy(m->d_order, order, N * 4, cudaMemcpyHostToDevice);
    float **bufs[] = {&m->d_p, &m->d_g, &m->d_m, &m->d_v, &m->d_mask};
    for (float **b : bufs)
        if ((e = cudaMalloc((void **)b, m->P * 4)) != cudaSuccess) return cleanup(mcuda(e, "made params"));
    cudaMemcpy(m->d_p, hp.data(), m->P * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->d_m, 0, m->P * 4);
    cudaMemset(m->d_v, 0, m->P * 4);
    cudaMemset(m->d_g, 0, m->P * 4);
    mk::k_masks<<<mk::nb(m->P, 256), 256>>>(m->d_mask, (int)N, (int)H, m->off_W1, m->off_W2,
                                             m->off_W3, m->P);
    mk::k_mul<<<mk::nb(m->P, 256), 256>>>(m->d_p, m->d_mask, m->P);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup(mcuda(e, "made masks"));
    if ((e = cudaMalloc((void **)&m->d_err, sizeof(int))) != cudaSuccess) return cleanup(mcuda(e, "made"));
    cudaMemset(m->d_err, 0, sizeof(int));
    if (l2_tc_supported((int)H)) {
        if ((e = cudaMalloc((void **)&m->d_w2b, H * H * 2)) != cudaSuccess)
            return cleanup(mcuda(e, "made BF16 weights"));
        if (!encode_bf16(&m->map_w2, m->d_w2b, (int64_t)H, (int)H, H > 256 ? 256 : (int)H))
            return cleanup(mfail(RTT_ERR_CUDA, "rtt_made_create: cuTensorMapEncodeTiled failed"));
        m->infer_bf16 = 1;
    }
    *out = m;
    return RTT_OK;
}

rtt_status rtt_made_destroy(rtt_made m) {
    if (!m) return RTT_OK;
    MGuard guard(m->device);
    cudaDeviceSynchronize();
    free_ws(m);
    cudaFree(m->d_order);
    cudaFree(m->d_p);
    cudaFree(m->d_g);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_mask);
    cudaFree(m->d_w2b);
    cudaFree(m->d_err);
    cudaFree(m->d_batch);
    cudaFree(m->d_fit);
    delete m;
    return RTT_OK;
}

rtt_status rtt_made_set_inference(rtt_made m, int32_t bf16) {
    if (!m) return mfail(RTT_ERR_INVALID_ARG, "rtt_made_set_inference: null model");
    if (bf16 && !m->d_w2b)
        return mfail(RTT_ERR_UNSUPPORTED, "rtt_made_set_inference: BF16 needs H in {64, 128, 192, "
                                          "256, 512}");
    m->infer_bf16 = bf16 ? 1 : 0;
    return RTT_OK;
}

rtt_status rtt_made_set_training(rtt_made m, int32_t tc) {
    if (!m) return mfail(RTT_ERR_INVALID_ARG, "rtt_made_set_training: null model");
    m->train_tc = tc ? 1 : 0;
    return RTT_OK;
}

rtt_status rtt_made_device_status(rtt_made m, int32_t *flags) {
    if (!m) return mfail(RTT_ERR_INVALID_ARG, "rtt_made_device_status: null model");
    MGuard guard(m->device);
    int v = 0;
    MC(cudaDeviceSynchronize(), "rtt_made_device_status");
    MC(cudaMemcpy(&v, m->d_err, sizeof(int), cudaMemcpyDeviceToHost), "rtt_made_device_status");
    MC(cudaMemset(m->d_err, 0, sizeof(int)), "rtt_made_device_status");
    if (flags) *flags = v;
    if (v & 1) return mfail(RTT_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel of the model expired");
    return RTT_OK;
}

rtt_status rtt_made_get_params(rtt_made m, float *host_out) {
    if (!m || !host_out) return mfail(RTT_ERR_INVALID_ARG, "rtt_made_get_params: null argument");
    MGuard guard(m->device);
    MC(cudaDeviceSynchronize(), "rtt_made_get_params");
    MC(cudaMemcpy(host_out, m->d_p, m->P * 4, cudaMemcpyDeviceToHost), "rtt_made_get_params");
    return RTT_OK;
}

rtt_status rtt_made_gradients(rtt_made m, const uint8_t *spins, int64_t B, float *grads,
                              double *nll, void *stream) {
    if (!m || !spins || !grads || B < 1) return mfail(RTT_ERR_INVALID_ARG, "rtt_made_gradients: bad arguments");
    MGuard guard(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    rtt_status s = ensure_ws(m, B);
    if (s != RTT_OK) return s;
    if ((s = gradients(m, spins, B, nll, st)) != RTT_OK) return s;
    MC(cudaMemcpyAsync(grads, m->d_g, m->P * 4, cudaMemcpyDeviceToDevice, st), "made grads copy");
    return RTT_OK;
}

// gradient of one batch and one Adam step (workspace already sized)
static rtt_status adam_step(rtt_made m, const uint8_t *spins, int64_t B, float lr, double *nll,
                            cudaStream_t st) {
    rtt_status s = gradients(m, spins, B, nll, st);
    if (s != RTT_OK) return s;
    m->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, (double)m->step));
    const float c2 = (float)(1.0 - pow(b2, (double)m->step));
    mk::k_adam<<<mk::nb(m->P, 256), 256, 0, st>>>(m->d_p, m->d_g, m->d_m, m->d_v, m->P, lr,
                                                   (float)b1, (float)b2, 1e-8f, c1, c2);
    MC(cudaGetLastError(), "made adam");
    return RTT_OK;
}

rtt_status rtt_made_train_step(rtt_made m, const uint8_t *spins, int64_t B, float lr, double *nll,
                               void *stream) {
    if (!m || !spins || B < 1 || !(lr > 0.f))
        return mfail(RTT_ERR_INVALID_ARG, "rtt_made_train_step: bad arguments");
    MGuard guard(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    rtt_status s = ensure_ws(m, B);
    if (s != RTT_OK) return s;
    return adam_step(m, spins, B, lr, nll, st);
}

rtt_status rtt_made_permutation(int64_t n, uint64_t seed, int64_t epoch, int64_t *host_out) {
    if (n < 1 || !host_out) return mfail(RTT_ERR_INVALID_ARG, "rtt_made_permutation: bad arguments");
    const mk::Shuffle sh = mk::shuffle_of((uint64_t)n, seed, epoch);
    for (int64_t i = 0; i < n; ++i) host_out[i] = (int64_t)mk::shuffle_index(sh, (uint64_t)i);
    return RTT_OK;
}

rtt_status rtt_made_fit(rtt_made m, const uint8_t *data, int64_t n, int32_t epochs, int32_t batch,
                        float lr, uint64_t shuffle_seed, double *nll_per_epoch, void *stream) {
    if (!m || !data || n < 1 || epochs < 0 || batch < 1 || batch > n || !(lr > 0.f))
        return mfail(RTT_ERR_INVALID_ARG, "rtt_made_fit: bad arguments");
    if (epochs == 0) return RTT_OK;
    MGuard guard(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    rtt_status s = ensure_ws(m, batch);
    if (s != RTT_OK) return s;
    if (batch > m->batch_cap || epochs > m->fit_cap) {
        MC(cudaStreamSynchronize(st), "made fit workspace");
        if (batch > m->batch_cap) {
            cudaFree(m->d_batch);
            m->d_batch = nullptr;
            m->batch_cap = 0;
            MC(cudaMalloc((void **)&m->d_batch, (size_t)batch * m->N), "made fit batch");
            m->batch_cap = batch;
        }
        if (epochs > m->fit_cap) {
            cudaFree(m->d_fit);
            m->d_fit = nullptr;
            m->fit_cap = 0;
            MC(cudaMalloc((void **)&m->d_fit, (size_t)(epochs + 1) * sizeof(double)), "made fit");
            m->fit_cap = epochs;
        }
    }
    MC(cudaMemsetAsync(m->d_fit, 0, (size_t)(epochs + 1) * sizeof(double), st), "made fit");
    double *batch_nll = m->d_fit + m->fit_cap;
    const int64_t n_batches = n / batch;
    for (int32_t e = 0; e < epochs; ++e) {
        const mk::Shuffle sh = mk::shuffle_of((uint64_t)n, shuffle_seed, e);
        for (int64_t b = 0; b < n_batches; ++b) {
            mk::k_gather_rows<<<(unsigned)batch, 128, 0, st>>>(data, sh, b * batch, batch, m->N,
                                                               m->d_batch);
            MC(cudaGetLastError(), "made fit gather");
            if ((s = adam_step(m, m->d_batch, batch, lr, batch_nll, st)) != RTT_OK) return s;
            mk::k_accumulate<<<1, 1, 0, st>>>(m->d_fit + e, batch_nll);
            MC(cudaGetLastError(), "made fit loss");
        }
    }
    if (nll_per_epoch) {
        MC(cudaMemcpyAsync(nll_per_epoch, m->d_fit, (size_t)epochs * sizeof(double),
                           cudaMemcpyDeviceToHost, st), "made fit loss copy");
        MC(cudaStreamSynchronize(st), "made fit");
        for (int32_t e = 0; e < epochs; ++e) nll_per_epoch[e] /= (double)n_batches;
    }
    return RTT_OK;
}

rtt_status rtt_made_log_prob(rtt_made m, const uint8_t *spins, int64_t B, double *logq, void *stream) {
    if (!m || !spins || !logq || B < 0) return mfail(RTT_ERR_INVALID_ARG, "rtt_made_log_prob: bad arguments");
    if (B == 0) return RTT_OK;
    MGuard guard(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    rtt_status s = ensure_ws(m, B);
    if (s != RTT_OK) return s;
    if (m->infer_bf16 && (s = refresh_w2(m, st)) != RTT_OK) return s;
    if ((s = forward_infer(m, spins, B, st)) != RTT_OK) return s;
    mk::k_loss<<<mk::nb(B, 128), 128, 0, st>>>(m->d_lg, spins, B, m->N, m->d_order, logq, nullptr);
    MC(cudaGetLastError(), "made log prob");
    return RTT_OK;
}

static rtt_status made_sample_into(rtt_made m, int64_t B, int64_t chain0, int64_t round,
                                   uint8_t *spins, double *logq, cudaStream_t st) {
    const int N = m->N, H = m->H;
    const float *p = m->d_p;
    // first-layer pre-activations start at the bias; x is not used here.  The
    // BF16 path keeps them and h2 feature-major ([H][B]) for coalesced access
    if (m->infer_bf16) {
        // per position: the layer on the tensor cores with the logit of position
        // d in its epilogue, the draw, then input d added to the feature-major
        // pre-activations together with the next BF16 operand
        mk::k_fill_T<<<mk::nb(B * H, 256), 256, 0, st>>>(m->d_dh1, B, H, p + m->off_b1);
        MC(cudaGetLastError(), "made sample init");
        const dim3 tb(32, 8), tg((unsigned)((B + 31) / 32), (unsigned)((H + 31) / 32));
        mk::k_relu_bf16_T<<<tg, tb, 0, st>>>(m->d_dh1, m->d_h1b, B, H);
        MC(cudaGetLastError(), "made sample layer 1 to BF16");
        for (int d = 0; d < N; ++d) {
            rtt_status s = layer2_tc(m, B, st, d);
            if (s != RTT_OK) return s;
            mk::k_sample_bit<<<mk::nb(B, 128), 128, 0, st>>>(d, B, N, m->d_lg, m->d_order, spins,
                                                              logq, m->d_x, m->seed, chain0, round);
            MC(cudaGetLastError(), "made sample position");
            if (d + 1 < N) {
                mk::k_h1_update_bf16_T<<<tg, tb, 0, st>>>(d, B, N, H, p + m->off_W1, m->d_x, m->d_dh1,
                                                          m->d_h1b);
                MC(cudaGetLastError(), "made sample update");
            }
        }
        return RTT_OK;
    }
    mk::k_fill_rows<<<mk::nb(B * H, 256), 256, 0, st>>>(m->d_dh1, B, H, p + m->off_b1);
    MC(cudaGetLastError(), "made sample init");
    for (int d = 0; d < N; ++d) {
        {
            mk::k_relu<<<mk::nb(B * H, 256), 256, 0, st>>>(m->d_dh1, m->d_h1, B * H);
            MC((mk::gemm<false, true>((int)B, H, H, m->d_h1, H, p + m->off_W2, H, m->d_h2, H,
                                      p + m->off_b2, 1, nullptr, nullptr, st)), "made sample layer 2");
        }
        mk::k_sample_pos<<<mk::nb(B, 128), 128, 0, st>>>(d, B, N, H, p + m->off_W1, p + m->off_W3,
                                                          p + m->off_b3, m->d_h2, m->d_dh1,
                                                          m->d_order, spins, logq, m->seed, chain0,
                                                          round);
        MC(cudaGetLastError(), "made sample position");
    }
    return RTT_OK;
}

rtt_status rtt_made_sample(rtt_made m, int64_t B, int64_t chain0, int64_t round, uint8_t *spins,
                           double *logq, void *stream) {
    if (!m || !spins || !logq || B < 0 || chain0 < 0 || round < 0)
        return mfail(RTT_ERR_INVALID_ARG, "rtt_made_sample: bad arguments");
    if (B == 0) return RTT_OK;
    MGuard guard(m->device);
    rtt_status s = ensure_ws(m, B);
    if (s != RTT_OK) return s;
    if (m->infer_bf16 && (s = refresh_w2(m, (cudaStream_t)stream)) != RTT_OK) return s;
    return made_sample_into(m, B, chain0, round, spins, logq, (cudaStream_t)stream);
}

rtt_status rtt_indep_mh(rtt_handle h, rtt_made m, uint8_t *spins, rtt_chain_state *state,
                        int64_t B, int64_t chain0, int64_t round, int64_t *n_accept, void *stream) {
    if (!h || !m || !spins || !state || B < 0 || chain0 < 0 || round < 0)
        return mfail(RTT_ERR_INVALID_ARG, "rtt_indep_mh: bad arguments");
    if (m->N != h->N) return mfail(RTT_ERR_INVALID_ARG, "rtt_indep_mh: model and state sizes differ");
    if (B == 0) return RTT_OK;
    MGuard guard(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    rtt_status s = ensure_ws(m, B);
    if (s != RTT_OK) return s;
    // log q(s) of the current configurations
    if (m->infer_bf16 && (s = refresh_w2(m, st)) != RTT_OK) return s;
    if ((s = forward_infer(m, spins, B, st)) != RTT_OK) return s;
    mk::k_loss<<<mk::nb(B, 128), 128, 0, st>>>(m->d_lg, spins, B, m->N, m->d_order, m->d_logq, nullptr);
    MC(cudaGetLastError(), "indep log q");
    // proposals s' ~ q with log q(s'), and psi(s')
    if ((s = made_sample_into(m, B, chain0, round, m->d_prop, m->d_plogq, st)) != RTT_OK) return s;
    if ((s = rtt_log_amplitudes(h, m->d_prop, B, nullptr, nullptr, m->d_pstate, stream)) != RTT_OK)
        return s;
    mk::k_indep_decide<<<mk::nb(B, 128), 128, 0, st>>>(B, m->N, spins, state, m->d_logq, m->d_prop,
                                                        m->d_pstate, m->d_plogq, m->seed, chain0,
                                                        round, n_accept);
    MC(cudaGetLastError(), "indep decide");
    return RTT_OK;
}

}  // extern "C"
