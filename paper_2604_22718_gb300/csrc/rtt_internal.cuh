// rtt_internal.cuh -- handle layout and device helpers shared by the library's
// translation units.  Not part of the public ABI (include/rtt.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "rtt.h"

// ----------------------------------------------------------------------------
// Handle
// ----------------------------------------------------------------------------
struct TcPlan;  // tensor-core operand forms (rtt_tc.cu)

struct rtt_s {
    int device = 0;
    int N = 0, L = 0, R = 0, chi = 0, chip = 0, n_bonds = 0;
    int precision = RTT_FP64;
    double J = 0, h = 0;
    uint64_t seed = 0;

    // device copies (owned)
    int32_t *d_q = nullptr;       // [N]    q[j] = path[j] (proposal order)
    int32_t *d_pos = nullptr;     // [N]    pos[i] = j with q[j] = i
    int32_t *d_bonds = nullptr;   // [n_bonds][2]
    // general (non-periodic) paths: site -> spin, last site of each spin, and
    // the first site the right stack holds (kmin) with its entry count nr
    bool periodic = true;
    int32_t *d_path = nullptr;    // [L]
    int32_t *d_last = nullptr;    // [N]
    int kmin = 0, nr = 0;
    std::vector<int32_t> bonds_host;  // the same on the host (lattice checks)
    void *d_A = nullptr;          // [L][2][chip][chip]  A_k[s][a][b]   (double or float)
    void *d_AT = nullptr;         // [L][2][chip][chip]  A_k[s][b][a]
    void *d_bl = nullptr;         // [chip]
    void *d_br = nullptr;         // [chip]
    TcPlan *tc = nullptr;         // BF16X3 forms

    // scratch (owned, grown on demand)
    int64_t cap_B = 0;
    void *d_lstack = nullptr;     // [B][N][chip]  left environments l_j, j < N
    int32_t *d_lexp = nullptr;    // [B][N]        cumulative exponents of l_j
    void *d_rstack = nullptr;     // [B][N][chip]  right environments r_{(R-1)N+1+q}
    int32_t *d_rexp = nullptr;    // [B][N]
    double *d_rows_mant = nullptr;   // [B][N+1]   psi(s^(path[j])) and psi(s) (j = N)
    int64_t *d_rows_exp = nullptr;   // [B][N+1]
    // the sampler's own environments (the local energy measured beside a
    // sweep uses the stacks above), and two snapshots of the spins entering
    // a measured sweep group
    void *d_sw_lstack = nullptr;  // [B][N][chip]
    int32_t *d_sw_lexp = nullptr; // [B][N]
    void *d_sw_rstack = nullptr;  // [B][N][chip]
    int32_t *d_sw_rexp = nullptr; // [B][N]
    uint8_t *d_snap[2] = {nullptr, nullptr};  // [B][N] each
    rtt_chain_state *d_amp = nullptr;         // [B] amplitudes for mixed energies

    // second stream on which the measured local energy runs beside the
    // sweeps, and its events (created with the handle)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_done[2] = {nullptr, nullptr};
    // third stream: the handle's sweep inside a dual step, so that the sweeps
    // of several states run side by side (each uses only its own sweep scratch)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_aux = nullptr;
    // dual step: this handle's amplitudes of its configurations are ready
    // (ev_amp), and the measurements run on its second stream are done (ev_meas)
    cudaEvent_t ev_amp = nullptr, ev_meas = nullptr;

    void *prof = nullptr;         // per-kernel event profiler (rtt_api.cu)

    size_t elem_bytes() const { return precision == RTT_FP64 ? 8 : 4; }
};

// Kernel kinds for the profiler.
enum RttKernel {
    KID_LEFT_ENV = 0, KID_RIGHT_ENV, KID_ROWS, KID_CHAIN_INIT, KID_SWEEP, KID_ELOC_REDUCE,
    KID_TC_LEFT_ENV, KID_TC_RIGHT_ENV, KID_TC_ROWS, KID_TC_CHAIN_INIT, KID_TC_SWEEP,
    KID_TC_SWEEP_ROWS, KID_COUNT
};
// Record the start / end of a kernel of kind `kid` on `st` (no-ops unless enabled).
void prof_begin(rtt_s *h, int kid, cudaStream_t st);
void prof_end(rtt_s *h, int kid, cudaStream_t st);

// thread-local last error message
void rtt_set_error(const std::string &msg);

// ----------------------------------------------------------------------------
// Launchers (SIMT FP64 / FP32), rtt_simt_f64.cu / rtt_simt_f32.cu
// ----------------------------------------------------------------------------
struct SimtArgs {
    const void *A, *AT, *bl, *br;
    const int32_t *q;
    int N, L, R, chip;
    const int32_t *p = nullptr;     // general path [L] (nullptr: periodic)
    const int32_t *last = nullptr;  // general path: last site of each spin [N]
    int kmin = 0;                   // general path: first site of the right stack
};

#define RTT_DECLARE_SIMT(SUFFIX)                                                                   \
    cudaError_t simt_left_env_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,         \
                                       void *lstack, int32_t *lexp, cudaStream_t st);              \
    cudaError_t simt_right_env_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,        \
                                        void *rstack, int32_t *rexp, cudaStream_t st);             \
    cudaError_t simt_rows_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,             \
                                   const void *lstack, const int32_t *lexp, const void *rstack,    \
                                   const int32_t *rexp, double *rows_mant, int64_t *rows_exp,      \
                                   cudaStream_t st);                                               \
    cudaError_t simt_chain_init_##SUFFIX(const SimtArgs &a, const uint8_t *spins, int64_t B,       \
                                         double *log_abs, int8_t *sign, rtt_chain_state *state,    \
                                         cudaStream_t st);                                         \
    cudaError_t simt_sweep_##SUFFIX(const SimtArgs &a, uint8_t *spins, rtt_chain_state *state,     \
                                    int64_t B, int64_t chain0, int64_t sweep0, int32_t n_sweeps,   \
                                    uint64_t seed, void *rstack, int32_t *rexp, void *lstack,      \
                                    int32_t *lexp, int64_t *n_accept, cudaStream_t st);

RTT_DECLARE_SIMT(f64)
RTT_DECLARE_SIMT(f32)

// ----------------------------------------------------------------------------
// Shared kernels (rtt_common.cu)
// ----------------------------------------------------------------------------
cudaError_t eloc_reduce(const uint8_t *spins, int64_t B, int N, const int32_t *pos,
                        const int32_t *bonds, int n_bonds, double J, double h,
                        const double *rows_mant, const int64_t *rows_exp, double *e_loc,
                        double *ratios, cudaStream_t st);
// Mixed local energy E^{ab} and ratio psi^b/psi^a from b's rows and a's amplitudes.
cudaError_t mixed_reduce(const uint8_t *spins, int64_t B, int N, const int32_t *pos,
                         const int32_t *bonds, int n_bonds, double J, double h,
                         const double *rows_mant, const int64_t *rows_exp,
                         const rtt_chain_state *amp_a, double *e_mixed, double *ratio,
                         cudaStream_t st);
cudaError_t launch_uniforms(uint64_t seed, int64_t n, const uint64_t *ctr, double *out,
                            cudaStream_t st);
cudaError_t stats_chain_means(const double *x, int T, int64_t B, double *chain_mean,
                              cudaStream_t st);
cudaError_t stats_lag_sums(const double *x, const double *chain_mean, int T, int64_t B, int lag0,
                           int nlag, double *acc, cudaStream_t st);
cudaError_t stats_bin_moments(const double *x, int T, int64_t B, int lb, double mean,
                              double *acc, cudaStream_t st);
cudaError_t stats_sum_i64(const int64_t *x, int64_t n, unsigned long long *out, cudaStream_t st);

// ----------------------------------------------------------------------------
// Tensor-core path (rtt_tc.cu)
// ----------------------------------------------------------------------------
rtt_status tc_plan_create(rtt_s *h, const double *tensors, const double *bl, const double *br);
void tc_plan_destroy(rtt_s *h);
rtt_status tc_left_env(rtt_s *h, const uint8_t *spins, int64_t B, cudaStream_t st);
rtt_status tc_right_env(rtt_s *h, const uint8_t *spins, int64_t B, cudaStream_t st);
rtt_status tc_rows(rtt_s *h, const uint8_t *spins, int64_t B, cudaStream_t st);
rtt_status tc_chain_init(rtt_s *h, const uint8_t *spins, int64_t B, double *log_abs, int8_t *sign,
                         rtt_chain_state *state, cudaStream_t st);
rtt_status tc_sweep(rtt_s *h, uint8_t *spins, rtt_chain_state *state, int64_t B, int64_t chain0,
                    int64_t sweep0, int32_t n_sweeps, int64_t *n_accept, cudaStream_t st);
bool tc_supported_chi(int chi);
// cuTensorMapEncodeTiled from the driver (null if unavailable); cast to its signature
void *tc_encode_tiled_fn();
int *tc_error_word(rtt_s *h);   // device error flags of the tensor-core kernels (or null)
rtt_status tc_wait_selftest(rtt_s *h, long long budget_cycles, cudaStream_t st);

// ----------------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------------
namespace rttd {

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds on a 4x64
// counter with two 64x64->128 products per round; the key is bumped by the
// golden-ratio / sqrt(3) Weyl constants before rounds 2..10.
__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B97F4A7C15ull;
            k1 += 0xBB67AE8584CAA73Bull;
        }
        const uint64_t p0h = __umul64hi(M0, c0), p0l = M0 * c0;
        const uint64_t p1h = __umul64hi(M1, c2), p1l = M1 * c2;
        const uint64_t n0 = p1h ^ c1 ^ k0, n2 = p0h ^ c3 ^ k1;
        c0 = n0;
        c1 = p1l;
        c2 = n2;
        c3 = p0l;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// Metropolis uniform in [0,1) with 53 random bits.
__device__ __forceinline__ double mcmc_uniform(uint64_t seed, uint64_t chain, uint64_t sweep,
                                               uint64_t proposal) {
    uint64_t x[4];
    philox4x64_10(chain, sweep, proposal, 0ull, seed, 0x4D434D43ull, x);
    return (double)(x[0] >> 11) * 0x1.0p-53;
}

// Exponent of a finite nonzero value, floor(log2|x|), from the IEEE fields.
__device__ __forceinline__ int exponent_of(double x) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    const int f = (int)((u >> 52) & 0x7ff);
    return f ? f - 1023 : ilogb(x);
}
__device__ __forceinline__ int exponent_of(float x) {
    const uint32_t u = __float_as_uint(x);
    const int f = (int)((u >> 23) & 0xff);
    return f ? f - 127 : ilogbf(x);
}

// x * 2^e, exact whenever the result is representable.
__device__ __forceinline__ double scale2(double x, int e) {
    if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
    return ldexp(x, e);
}
__device__ __forceinline__ float scale2(float x, int e) {
    if (e >= -126 && e <= 127) return x * __uint_as_float((uint32_t)(e + 127) << 23);
    return ldexpf(x, e);
}

// Whether 2^e is a normal number of x's type, and that power itself.
__device__ __forceinline__ bool pow2_normal(double, int e) { return e >= -1022 && e <= 1023; }
__device__ __forceinline__ bool pow2_normal(float, int e) { return e >= -126 && e <= 127; }
__device__ __forceinline__ double pow2(double, int e) {
    return __longlong_as_double((long long)(e + 1023) << 52);
}
__device__ __forceinline__ float pow2(float, int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

}  // namespace rttd

#define RTT_CUDA_TRY(expr)                                                                         \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return _e;                                                          \
    } while (0)
