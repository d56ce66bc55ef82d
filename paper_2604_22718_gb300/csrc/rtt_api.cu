// rtt_api.cu -- the C ABI declared in include/rtt.h: handle lifecycle,
// argument validation, scratch management and dispatch to the SIMT (FP64,
// FP32) and tensor-core (BF16X3) kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rtt_internal.cuh"

namespace {

thread_local std::string g_last_error;

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

rtt_status fail(rtt_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

rtt_status cuda_fail(cudaError_t e, const char *where) {
    return fail(e == cudaErrorMemoryAllocation ? RTT_ERR_OOM : RTT_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define API_CUDA(expr, where)                                                                      \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return cuda_fail(_e, where);                                        \
    } while (0)

// As API_CUDA inside rtt_create, where a failure also frees the handle.
#define API_CUDA_CLEANUP(expr, where)                                                              \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return cleanup(cuda_fail(_e, where));                               \
    } while (0)

int padded_chi(int chi) {
    int p = 1;
    while (p < chi) p <<= 1;
    return p;
}

template <typename T>
void pack_tensors(const double *src, int L, int chi, int chip, std::vector<T> &A,
                  std::vector<T> &AT) {
    const size_t plane = (size_t)chip * chip;
    A.assign((size_t)L * 2 * plane, T(0));
    AT.assign((size_t)L * 2 * plane, T(0));
    for (int k = 0; k < L; ++k)
        for (int s = 0; s < 2; ++s)
            for (int a = 0; a < chi; ++a)
                for (int b = 0; b < chi; ++b) {
                    const double v = src[(((size_t)k * 2 + s) * chi + a) * chi + b];
                    A[((size_t)k * 2 + s) * plane + (size_t)a * chip + b] = (T)v;
                    AT[((size_t)k * 2 + s) * plane + (size_t)b * chip + a] = (T)v;
                }
}

template <typename T>
rtt_status upload(const std::vector<T> &v, void **dst, const char *what) {
    API_CUDA(cudaMalloc(dst, v.size() * sizeof(T)), what);
    API_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return RTT_OK;
}

void free_scratch(rtt_s *h) {
    cudaFree(h->d_lstack);
    cudaFree(h->d_lexp);
    cudaFree(h->d_rstack);
    cudaFree(h->d_rexp);
    cudaFree(h->d_rows_mant);
    cudaFree(h->d_rows_exp);
    cudaFree(h->d_sw_lstack);
    cudaFree(h->d_sw_lexp);
    cudaFree(h->d_sw_rstack);
    cudaFree(h->d_sw_rexp);
    cudaFree(h->d_snap[0]);
    cudaFree(h->d_snap[1]);
    cudaFree(h->d_amp);
    h->d_amp = nullptr;
    h->d_lstack = h->d_rstack = nullptr;
    h->d_lexp = h->d_rexp = nullptr;
    h->d_rows_mant = nullptr;
    h->d_rows_exp = nullptr;
    h->d_sw_lstack = h->d_sw_rstack = nullptr;
    h->d_sw_lexp = h->d_sw_rexp = nullptr;
    h->d_snap[0] = h->d_snap[1] = nullptr;
    h->cap_B = 0;
}

size_t scratch_bytes_for(const rtt_s *h, int64_t B) {
    const size_t per = h->chip * h->elem_bytes() + 4;  // one environment entry and its exponent
    // left (N entries) and right (nr entries) stacks, for the energy and for the sampler
    const size_t stacks = 2 * (size_t)B * (h->N + h->nr) * per;
    const size_t rows = (size_t)B * (h->N + 1) * 16;
    const size_t snap = (size_t)B * h->N;
    return stacks + rows + 2 * snap + (size_t)B * sizeof(rtt_chain_state);
}

rtt_status ensure_scratch(rtt_s *h, int64_t B) {
    if (B <= h->cap_B) return RTT_OK;
    API_CUDA(cudaDeviceSynchronize(), "scratch resize (sync)");
    free_scratch(h);
    const size_t eb = h->elem_bytes();
    const size_t nv = (size_t)B * h->N;
    API_CUDA(cudaMalloc(&h->d_lstack, nv * h->chip * eb), "scratch l-stack");
    API_CUDA(cudaMalloc((void **)&h->d_lexp, nv * 4), "scratch l-exp");
    const size_t nvr = (size_t)B * h->nr;  // right stacks: nr entries per chain
    API_CUDA(cudaMalloc(&h->d_rstack, nvr * h->chip * eb), "scratch r-stack");
    API_CUDA(cudaMalloc((void **)&h->d_rexp, nvr * 4), "scratch r-exp");
    API_CUDA(cudaMalloc((void **)&h->d_rows_mant, (size_t)B * (h->N + 1) * 8), "scratch rows");
    API_CUDA(cudaMalloc((void **)&h->d_rows_exp, (size_t)B * (h->N + 1) * 8), "scratch rows");
    API_CUDA(cudaMalloc(&h->d_sw_lstack, nv * h->chip * eb), "scratch sweep l-stack");
    API_CUDA(cudaMalloc((void **)&h->d_sw_lexp, nv * 4), "scratch sweep l-exp");
    API_CUDA(cudaMalloc(&h->d_sw_rstack, nvr * h->chip * eb), "scratch sweep r-stack");
    API_CUDA(cudaMalloc((void **)&h->d_sw_rexp, nvr * 4), "scratch sweep r-exp");
    API_CUDA(cudaMalloc((void **)&h->d_snap[0], nv), "scratch spin snapshot");
    API_CUDA(cudaMalloc((void **)&h->d_snap[1], nv), "scratch spin snapshot");
    API_CUDA(cudaMalloc((void **)&h->d_amp, (size_t)B * sizeof(rtt_chain_state)), "scratch amplitudes");
    h->cap_B = B;
    return RTT_OK;
}

SimtArgs simt_args(const rtt_s *h) {
    SimtArgs a{h->d_A, h->d_AT, h->d_bl, h->d_br, h->d_q, h->N, h->L, h->R, h->chip};
    if (!h->periodic) {
        a.p = h->d_path;
        a.last = h->d_last;
        a.kmin = h->kmin;
    }
    return a;
}

rtt_status check_handle(rtt_handle h) {
    if (!h) return fail(RTT_ERR_INVALID_ARG, "null handle");
    return RTT_OK;
}

// Environments + rows + reduction for the spins currently in `spins`.
// If `have_left` the left stack already holds l_j for these spins.
// Environments and flip rows (psi(s^(path[j])) and psi(s)) for the spins in
// `spins`, into the handle's rows.  If `have_left` the left stack already holds
// l_j for these spins.
rtt_status rows_pipeline(rtt_s *h, const uint8_t *spins, int64_t B, bool have_left,
                         cudaStream_t st) {
    if (h->precision >= RTT_BF16X3) {
        rtt_status s;
        if (!have_left && (s = tc_left_env(h, spins, B, st)) != RTT_OK) return s;
        if ((s = tc_right_env(h, spins, B, st)) != RTT_OK) return s;
        if ((s = tc_rows(h, spins, B, st)) != RTT_OK) return s;
    } else {
        const SimtArgs a = simt_args(h);
        const bool f64 = h->precision == RTT_FP64;
        if (!have_left) {
            prof_begin(h, KID_LEFT_ENV, st);
            API_CUDA(f64 ? simt_left_env_f64(a, spins, B, h->d_lstack, h->d_lexp, st)
                         : simt_left_env_f32(a, spins, B, h->d_lstack, h->d_lexp, st),
                     "left environments");
            prof_end(h, KID_LEFT_ENV, st);
        }
        prof_begin(h, KID_RIGHT_ENV, st);
        API_CUDA(f64 ? simt_right_env_f64(a, spins, B, h->d_rstack, h->d_rexp, st)
                     : simt_right_env_f32(a, spins, B, h->d_rstack, h->d_rexp, st),
                 "right environments");
        prof_end(h, KID_RIGHT_ENV, st);
        prof_begin(h, KID_ROWS, st);
        API_CUDA(f64 ? simt_rows_f64(a, spins, B, h->d_lstack, h->d_lexp, h->d_rstack, h->d_rexp,
                                     h->d_rows_mant, h->d_rows_exp, st)
                     : simt_rows_f32(a, spins, B, h->d_lstack, h->d_lexp, h->d_rstack, h->d_rexp,
                                     h->d_rows_mant, h->d_rows_exp, st),
                 "flip rows");
        prof_end(h, KID_ROWS, st);
    }
    return RTT_OK;
}

rtt_status energy_pipeline(rtt_s *h, const uint8_t *spins, int64_t B, double *e_loc,
                           double *ratios, bool have_left, cudaStream_t st) {
    rtt_status s = rows_pipeline(h, spins, B, have_left, st);
    if (s != RTT_OK) return s;
    prof_begin(h, KID_ELOC_REDUCE, st);
    API_CUDA(eloc_reduce(spins, B, h->N, h->d_pos, h->d_bonds, h->n_bonds, h->J, h->h,
                         h->d_rows_mant, h->d_rows_exp, e_loc, ratios, st),
             "local-energy reduction");
    prof_end(h, KID_ELOC_REDUCE, st);
    return RTT_OK;
}

const char *kKernelNames[KID_COUNT] = {
    "simt_left_env", "simt_right_env", "simt_rows", "simt_chain_init", "simt_sweep",
    "eloc_reduce", "tc_left_env", "tc_right_env", "tc_rows", "tc_chain_init", "tc_sweep",
    "tc_sweep_rows"};

struct Profiler {
    bool on = false;
    struct Rec {
        int kid;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open_ev = nullptr;
    double ms[KID_COUNT] = {0};
    int64_t n[KID_COUNT] = {0};
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void reset() {
        for (auto &r : pending) {
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
        for (int k = 0; k < KID_COUNT; ++k) {
            ms[k] = 0;
            n[k] = 0;
        }
    }
    ~Profiler() {
        reset();
        for (auto e : pool) cudaEventDestroy(e);
    }
};

Profiler *prof_of(rtt_s *h) {
    if (!h->prof) h->prof = new Profiler();
    return (Profiler *)h->prof;
}

}  // namespace

void prof_begin(rtt_s *h, int kid, cudaStream_t st) {
    if (!h->prof || !((Profiler *)h->prof)->on) return;
    Profiler *p = (Profiler *)h->prof;
    p->open_ev = p->get();
    cudaEventRecord(p->open_ev, st);
    (void)kid;
}

void prof_end(rtt_s *h, int kid, cudaStream_t st) {
    if (!h->prof || !((Profiler *)h->prof)->on || !((Profiler *)h->prof)->open_ev) return;
    Profiler *p = (Profiler *)h->prof;
    cudaEvent_t b = p->get();
    cudaEventRecord(b, st);
    p->pending.push_back({kid, p->open_ev, b});
    p->open_ev = nullptr;
}

void rtt_set_error(const std::string &msg) { g_last_error = msg; }

extern "C" {

const char *rtt_last_error(void) { return g_last_error.c_str(); }

const char *rtt_status_string(rtt_status s) {
    switch (s) {
        case RTT_OK: return "RTT_OK";
        case RTT_ERR_INVALID_ARG: return "RTT_ERR_INVALID_ARG";
        case RTT_ERR_CUDA: return "RTT_ERR_CUDA";
        case RTT_ERR_OOM: return "RTT_ERR_OOM";
        case RTT_ERR_NUMERIC: return "RTT_ERR_NUMERIC";
        case RTT_ERR_TIMEOUT: return "RTT_ERR_TIMEOUT";
        case RTT_ERR_UNSUPPORTED: return "RTT_ERR_UNSUPPORTED";
    }
    return "RTT_ERR_UNKNOWN";
}

rtt_status rtt_create(const rtt_desc *d, rtt_handle *out) {
    g_last_error.clear();
    if (!d || !out) return fail(RTT_ERR_INVALID_ARG, "rtt_create: null desc or out");
    *out = nullptr;
    if (d->n_spins < 1 || d->length < 1 || d->chi < 1)
        return fail(RTT_ERR_INVALID_ARG, "rtt_create: n_spins, length and chi must be >= 1");
    if (d->chi > 256) return fail(RTT_ERR_UNSUPPORTED, "rtt_create: chi > 256");
    if (!d->path || !d->tensors || !d->b_left || !d->b_right)
        return fail(RTT_ERR_INVALID_ARG, "rtt_create: null path/tensors/boundary");
    if (d->n_bonds < 0 || (d->n_bonds > 0 && !d->bonds))
        return fail(RTT_ERR_INVALID_ARG, "rtt_create: bad bonds");
    if (d->precision < RTT_FP64 || d->precision > RTT_FP16X3)
        return fail(RTT_ERR_INVALID_ARG, "rtt_create: unknown precision");
    const int N = d->n_spins, L = d->length, chi = d->chi;
    for (int k = 0; k < L; ++k)
        if (d->path[k] < 0 || d->path[k] >= N)
            return fail(RTT_ERR_INVALID_ARG, "rtt_create: path entry out of range");
    for (int q = 0; q < 2 * d->n_bonds; ++q)
        if (d->bonds[q] < 0 || d->bonds[q] >= N)
            return fail(RTT_ERR_INVALID_ARG, "rtt_create: bond index out of range");
    for (int q = 0; q < d->n_bonds; ++q)
        if (d->bonds[2 * q] == d->bonds[2 * q + 1])
            return fail(RTT_ERR_INVALID_ARG, "rtt_create: bond joins a spin to itself");
    // periodic path: block 0 a permutation, path[k] = path[k mod N]
    if (L % N != 0) return fail(RTT_ERR_UNSUPPORTED, "rtt_create: length is not a multiple of N");
    std::vector<int32_t> pos(N, -1);
    for (int j = 0; j < N; ++j) {
        if (pos[d->path[j]] >= 0)
            return fail(RTT_ERR_UNSUPPORTED, "rtt_create: first N sites are not a permutation");
        pos[d->path[j]] = j;
    }
    bool periodic = true;
    for (int k = N; k < L; ++k)
        if (d->path[k] != d->path[k % N]) periodic = false;
    // last site of every spin, and the first site the right stacks must hold
    std::vector<int32_t> last(N, -1);
    for (int k = 0; k < L; ++k) last[d->path[k]] = k;
    int kmin = L;
    for (int i = 0; i < N; ++i) kmin = std::min(kmin, last[i] + 1);
    const size_t nt = (size_t)L * 2 * chi * chi;
    for (size_t t = 0; t < nt; ++t)
        if (!isfinite(d->tensors[t])) return fail(RTT_ERR_NUMERIC, "rtt_create: non-finite tensor entry");
    for (int a = 0; a < chi; ++a)
        if (!isfinite(d->b_left[a]) || !isfinite(d->b_right[a]))
            return fail(RTT_ERR_NUMERIC, "rtt_create: non-finite boundary entry");
    const bool tensor_core = d->precision == RTT_BF16X3 || d->precision == RTT_FP16X3;
    if (tensor_core && !tc_supported_chi(chi))
        return fail(RTT_ERR_UNSUPPORTED, "rtt_create: BF16X3/FP16X3 need chi in {64,128}");

    int dev = d->device;
    if (dev < 0) API_CUDA(cudaGetDevice(&dev), "rtt_create: cudaGetDevice");
    DeviceGuard guard(dev);
    rtt_s *h = new rtt_s();
    h->device = dev;
    h->N = N;
    h->L = L;
    h->R = L / N;
    h->chi = chi;
    h->chip = padded_chi(chi);
    h->n_bonds = d->n_bonds;
    h->periodic = periodic;
    h->kmin = kmin;
    h->nr = L - kmin + 1;
    h->precision = d->precision;
    h->J = d->J;
    h->h = d->h;
    h->seed = d->seed;
    auto cleanup = [&](rtt_status s) {
        rtt_destroy(h);
        return s;
    };
    rtt_status s;
    API_CUDA_CLEANUP(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking),
                     "rtt_create: second stream");
    API_CUDA_CLEANUP(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking),
                     "rtt_create: third stream");
    API_CUDA_CLEANUP(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "rtt_create: events");
    API_CUDA_CLEANUP(cudaEventCreateWithFlags(&h->ev_aux, cudaEventDisableTiming), "rtt_create: events");
    API_CUDA_CLEANUP(cudaEventCreateWithFlags(&h->ev_amp, cudaEventDisableTiming), "rtt_create: events");
    API_CUDA_CLEANUP(cudaEventCreateWithFlags(&h->ev_meas, cudaEventDisableTiming), "rtt_create: events");
    for (int i = 0; i < 2; ++i)
        API_CUDA_CLEANUP(cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming),
                         "rtt_create: events");
    std::vector<int32_t> q(d->path, d->path + N);
    if ((s = upload(q, (void **)&h->d_q, "rtt_create: path")) != RTT_OK) return cleanup(s);
    if ((s = upload(pos, (void **)&h->d_pos, "rtt_create: positions")) != RTT_OK) return cleanup(s);
    if (!periodic) {
        std::vector<int32_t> path(d->path, d->path + L);
        if ((s = upload(path, (void **)&h->d_path, "rtt_create: path")) != RTT_OK) return cleanup(s);
        if ((s = upload(last, (void **)&h->d_last, "rtt_create: last sites")) != RTT_OK)
            return cleanup(s);
    }
    std::vector<int32_t> bonds(d->bonds, d->bonds + 2 * d->n_bonds);
    h->bonds_host = bonds;
    if (bonds.empty()) bonds.push_back(0);
    if ((s = upload(bonds, (void **)&h->d_bonds, "rtt_create: bonds")) != RTT_OK) return cleanup(s);
    const int chip = h->chip;
    if (d->precision == RTT_FP64) {
        std::vector<double> A, AT, bl(chip, 0.0), br(chip, 0.0);
        pack_tensors<double>(d->tensors, L, chi, chip, A, AT);
        std::copy(d->b_left, d->b_left + chi, bl.begin());
        std::copy(d->b_right, d->b_right + chi, br.begin());
        if ((s = upload(A, &h->d_A, "rtt_create: tensors")) != RTT_OK) return cleanup(s);
        if ((s = upload(AT, &h->d_AT, "rtt_create: tensors^T")) != RTT_OK) return cleanup(s);
        if ((s = upload(bl, &h->d_bl, "rtt_create: b_L")) != RTT_OK) return cleanup(s);
        if ((s = upload(br, &h->d_br, "rtt_create: b_R")) != RTT_OK) return cleanup(s);
    } else if (d->precision == RTT_FP32) {
        std::vector<float> A, AT, bl(chip, 0.f), br(chip, 0.f);
        pack_tensors<float>(d->tensors, L, chi, chip, A, AT);
        for (int a = 0; a < chi; ++a) {
            bl[a] = (float)d->b_left[a];
            br[a] = (float)d->b_right[a];
        }
        if ((s = upload(A, &h->d_A, "rtt_create: tensors")) != RTT_OK) return cleanup(s);
        if ((s = upload(AT, &h->d_AT, "rtt_create: tensors^T")) != RTT_OK) return cleanup(s);
        if ((s = upload(bl, &h->d_bl, "rtt_create: b_L")) != RTT_OK) return cleanup(s);
        if ((s = upload(br, &h->d_br, "rtt_create: b_R")) != RTT_OK) return cleanup(s);
    } else {
        if ((s = tc_plan_create(h, d->tensors, d->b_left, d->b_right)) != RTT_OK) return cleanup(s);
    }
    *out = h;
    return RTT_OK;
}

rtt_status rtt_destroy(rtt_handle h) {
    if (!h) return RTT_OK;
    DeviceGuard guard(h->device);
    cudaDeviceSynchronize();
    free_scratch(h);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_aux) cudaEventDestroy(h->ev_aux);
    if (h->ev_amp) cudaEventDestroy(h->ev_amp);
    if (h->ev_meas) cudaEventDestroy(h->ev_meas);
    for (int i = 0; i < 2; ++i)
        if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
    tc_plan_destroy(h);
    delete (Profiler *)h->prof;
    h->prof = nullptr;
    cudaFree(h->d_q);
    cudaFree(h->d_pos);
    cudaFree(h->d_bonds);
    cudaFree(h->d_path);
    cudaFree(h->d_last);
    cudaFree(h->d_A);
    cudaFree(h->d_AT);
    cudaFree(h->d_bl);
    cudaFree(h->d_br);
    delete h;
    return RTT_OK;
}

rtt_status rtt_reserve(rtt_handle h, int64_t B) {
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (B < 0) return fail(RTT_ERR_INVALID_ARG, "rtt_reserve: B < 0");
    DeviceGuard guard(h->device);
    return ensure_scratch(h, B);
}

rtt_status rtt_scratch_bytes(rtt_handle h, int64_t B, size_t *bytes) {
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (!bytes || B < 0) return fail(RTT_ERR_INVALID_ARG, "rtt_scratch_bytes: bad arguments");
    *bytes = scratch_bytes_for(h, B);
    return RTT_OK;
}

rtt_status rtt_log_amplitudes(rtt_handle h, const uint8_t *spins, int64_t B, double *log_abs,
                              int8_t *sign, rtt_chain_state *state, void *stream) {
    g_last_error.clear();
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (B < 0) return fail(RTT_ERR_INVALID_ARG, "rtt_log_amplitudes: B < 0");
    if (B == 0) return RTT_OK;
    if (!spins) return fail(RTT_ERR_INVALID_ARG, "rtt_log_amplitudes: null spins");
    if (!log_abs && !sign && !state)
        return fail(RTT_ERR_INVALID_ARG, "rtt_log_amplitudes: no output requested");
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaGetLastError(), "rtt_log_amplitudes: pending error");
    if (h->precision >= RTT_BF16X3) return tc_chain_init(h, spins, B, log_abs, sign, state, st);
    const SimtArgs a = simt_args(h);
    prof_begin(h, KID_CHAIN_INIT, st);
    API_CUDA(h->precision == RTT_FP64 ? simt_chain_init_f64(a, spins, B, log_abs, sign, state, st)
                                      : simt_chain_init_f32(a, spins, B, log_abs, sign, state, st),
             "rtt_log_amplitudes");
    prof_end(h, KID_CHAIN_INIT, st);
    return RTT_OK;
}

rtt_status rtt_local_energy(rtt_handle h, const uint8_t *spins, int64_t B, double *e_loc,
                            double *ratios, void *stream) {
    g_last_error.clear();
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (B < 0) return fail(RTT_ERR_INVALID_ARG, "rtt_local_energy: B < 0");
    if (B == 0) return RTT_OK;
    if (!spins || !e_loc) return fail(RTT_ERR_INVALID_ARG, "rtt_local_energy: null spins or e_loc");
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaGetLastError(), "rtt_local_energy: pending error");
    if ((s = ensure_scratch(h, B)) != RTT_OK) return s;
    return energy_pipeline(h, spins, B, e_loc, ratios, false, st);
}

namespace {
// psi^a of the configurations into a's amplitude scratch, on stream st.
rtt_status mixed_amplitudes(rtt_s *a, const uint8_t *spins, int64_t B, cudaStream_t st) {
    rtt_status s;
    if (a->precision >= RTT_BF16X3) {
        if ((s = tc_chain_init(a, spins, B, nullptr, nullptr, a->d_amp, st)) != RTT_OK) return s;
    } else {
        const SimtArgs sa = simt_args(a);
        prof_begin(a, KID_CHAIN_INIT, st);
        API_CUDA(a->precision == RTT_FP64
                     ? simt_chain_init_f64(sa, spins, B, nullptr, nullptr, a->d_amp, st)
                     : simt_chain_init_f32(sa, spins, B, nullptr, nullptr, a->d_amp, st),
                 "mixed local energy: amplitudes");
        prof_end(a, KID_CHAIN_INIT, st);
    }
    return RTT_OK;
}

// E^{ab} and r^{ab} from b's flip rows and a's amplitudes (already computed).
rtt_status mixed_rows(rtt_s *a, rtt_s *b, const uint8_t *spins, int64_t B, double *e_mixed,
                      double *ratio, cudaStream_t st) {
    rtt_status s;
    if ((s = rows_pipeline(b, spins, B, false, st)) != RTT_OK) return s;
    prof_begin(b, KID_ELOC_REDUCE, st);
    API_CUDA(mixed_reduce(spins, B, b->N, b->d_pos, b->d_bonds, b->n_bonds, b->J, b->h,
                          b->d_rows_mant, b->d_rows_exp, a->d_amp, e_mixed, ratio, st),
             "mixed local energy: reduction");
    prof_end(b, KID_ELOC_REDUCE, st);
    return RTT_OK;
}

rtt_status same_lattice(const rtt_s *a, const rtt_s *b, const char *where) {
    if (a->device != b->device)
        return fail(RTT_ERR_INVALID_ARG, std::string(where) + ": handles on different devices");
    if (a->N != b->N || a->n_bonds != b->n_bonds || a->bonds_host != b->bonds_host ||
        a->J != b->J || a->h != b->h)
        return fail(RTT_ERR_INVALID_ARG, std::string(where) + ": handles differ in N, bonds, J or h");
    return RTT_OK;
}
}  // namespace

rtt_status rtt_dual_step(const rtt_handle *handles, int32_t M, uint8_t *const *spins,
                         rtt_chain_state *const *state, int64_t B, int64_t chain0, int64_t sweep,
                         double *e_mixed, double *ratio, int64_t *const *n_accept, void *stream) {
    g_last_error.clear();
    if (!handles || M < 1 || !spins || !state)
        return fail(RTT_ERR_INVALID_ARG, "rtt_dual_step: null argument or M < 1");
    if (B < 0 || chain0 < 0 || sweep < 0)
        return fail(RTT_ERR_INVALID_ARG, "rtt_dual_step: negative B, chain0 or sweep");
    for (int m = 0; m < M; ++m) {
        if (!handles[m]) return fail(RTT_ERR_INVALID_ARG, "rtt_dual_step: null handle");
        for (int m2 = 0; m2 < m; ++m2)
            if (handles[m2] == handles[m])
                return fail(RTT_ERR_INVALID_ARG, "rtt_dual_step: a handle appears twice");
        rtt_status s = same_lattice(handles[0], handles[m], "rtt_dual_step");
        if (s != RTT_OK) return s;
        if (B > 0 && (!spins[m] || !state[m]))
            return fail(RTT_ERR_INVALID_ARG, "rtt_dual_step: null spins or state");
    }
    if (B == 0) return RTT_OK;
    rtt_s *h0 = handles[0];
    DeviceGuard guard(h0->device);
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaGetLastError(), "rtt_dual_step: pending error");
    rtt_status s;
    for (int m = 0; m < M; ++m)
        if ((s = ensure_scratch(handles[m], B)) != RTT_OK) return s;
    const size_t nv = (size_t)B * h0->N;
    const bool meas = e_mixed || ratio;
    // snapshots of the entering configurations, and a's amplitudes of them on
    // a's second stream
    for (int a = 0; a < M; ++a) {
        rtt_s *ha = handles[a];
        if (meas)
            API_CUDA(cudaMemcpyAsync(ha->d_snap[0], spins[a], nv, cudaMemcpyDeviceToDevice, st),
                     "rtt_dual_step: spin snapshot");
        API_CUDA(cudaEventRecord(ha->ev_fork, st), "rtt_dual_step: fork");
        if (meas) {
            API_CUDA(cudaStreamWaitEvent(ha->side, ha->ev_fork, 0), "rtt_dual_step: fork");
            if ((s = mixed_amplitudes(ha, ha->d_snap[0], B, ha->side)) != RTT_OK) return s;
            API_CUDA(cudaEventRecord(ha->ev_amp, ha->side), "rtt_dual_step: amplitudes");
        }
    }
    // the pairs (a, b) in M waves: wave w takes b = (a + w) mod M for every a, so
    // within a wave each b -- whose energy scratch the pair uses -- appears once;
    // pair (a, b) runs on b's second stream after a's amplitudes
    if (meas) {
        for (int w = 0; w < M; ++w)
            for (int a = 0; a < M; ++a) {
                const int b = (a + w) % M;
                rtt_s *ha = handles[a], *hb = handles[b];
                if (b != a)
                    API_CUDA(cudaStreamWaitEvent(hb->side, ha->ev_amp, 0), "rtt_dual_step: wave");
                const size_t off = ((size_t)a * M + b) * B;
                if ((s = mixed_rows(ha, hb, ha->d_snap[0], B, e_mixed ? e_mixed + off : nullptr,
                                    ratio ? ratio + off : nullptr, hb->side)) != RTT_OK)
                    return s;
            }
        for (int b = 0; b < M; ++b)
            API_CUDA(cudaEventRecord(handles[b]->ev_meas, handles[b]->side), "rtt_dual_step: join");
    }
    for (int a = 0; a < M; ++a) {
        rtt_s *ha = handles[a];
        // one sweep of a's chains, after the snapshot.  A SIMT sweep holds few
        // SMs (one thread group per chain), so it runs on a's third stream beside
        // the other states' sweeps (each uses its own sweep scratch); a
        // tensor-core sweep fills 64 SMs per 4096 chains and stays in the
        // caller's stream, leaving the other SMs to the measurements
        cudaStream_t sa_st = ha->precision >= RTT_BF16X3 ? st : ha->aux;
        API_CUDA(cudaStreamWaitEvent(sa_st, ha->ev_fork, 0), "rtt_dual_step: fork");
        if (ha->precision >= RTT_BF16X3) {
            if ((s = tc_sweep(ha, spins[a], state[a], B, chain0, sweep, 1,
                              n_accept ? n_accept[a] : nullptr, sa_st)) != RTT_OK)
                return s;
        } else {
            const SimtArgs sa = simt_args(ha);
            prof_begin(ha, KID_SWEEP, sa_st);
            API_CUDA(ha->precision == RTT_FP64
                         ? simt_sweep_f64(sa, spins[a], state[a], B, chain0, sweep, 1, ha->seed,
                                          ha->d_sw_rstack, ha->d_sw_rexp, nullptr, nullptr,
                                          n_accept ? n_accept[a] : nullptr, sa_st)
                         : simt_sweep_f32(sa, spins[a], state[a], B, chain0, sweep, 1, ha->seed,
                                          ha->d_sw_rstack, ha->d_sw_rexp, nullptr, nullptr,
                                          n_accept ? n_accept[a] : nullptr, sa_st),
                     "rtt_dual_step: sweep kernel");
            prof_end(ha, KID_SWEEP, sa_st);
        }
        API_CUDA(cudaEventRecord(ha->ev_aux, sa_st), "rtt_dual_step: join");
    }
    // the caller's stream waits for every sweep and every measurement stream
    for (int a = 0; a < M; ++a) {
        API_CUDA(cudaStreamWaitEvent(st, handles[a]->ev_aux, 0), "rtt_dual_step: join");
        if (meas)
            API_CUDA(cudaStreamWaitEvent(st, handles[a]->ev_meas, 0), "rtt_dual_step: join");
    }
    return RTT_OK;
}

rtt_status rtt_mixed_local_energy(rtt_handle a, rtt_handle b, const uint8_t *spins, int64_t B,
                                  double *e_mixed, double *ratio, void *stream) {
    g_last_error.clear();
    if (!a || !b) return fail(RTT_ERR_INVALID_ARG, "rtt_mixed_local_energy: null handle");
    if (B < 0) return fail(RTT_ERR_INVALID_ARG, "rtt_mixed_local_energy: B < 0");
    rtt_status s = same_lattice(a, b, "rtt_mixed_local_energy");
    if (s != RTT_OK) return s;
    if (B == 0) return RTT_OK;
    if (!spins || !e_mixed)
        return fail(RTT_ERR_INVALID_ARG, "rtt_mixed_local_energy: null spins or e_mixed");
    DeviceGuard guard(a->device);
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaGetLastError(), "rtt_mixed_local_energy: pending error");
    if ((s = ensure_scratch(a, B)) != RTT_OK) return s;
    if ((s = ensure_scratch(b, B)) != RTT_OK) return s;
    if ((s = mixed_amplitudes(a, spins, B, st)) != RTT_OK) return s;
    return mixed_rows(a, b, spins, B, e_mixed, ratio, st);
}

rtt_status rtt_mcmc_sweep(rtt_handle h, uint8_t *spins, rtt_chain_state *state, int64_t B,
                          int64_t chain0, int64_t sweep0, int32_t n_sweeps, int32_t measure_every,
                          double *e_loc_trace, int64_t *n_accept, void *stream) {
    g_last_error.clear();
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (B < 0 || n_sweeps < 0 || chain0 < 0 || sweep0 < 0)
        return fail(RTT_ERR_INVALID_ARG, "rtt_mcmc_sweep: negative B, chain0, sweep0 or n_sweeps");
    if (e_loc_trace && measure_every < 1)
        return fail(RTT_ERR_INVALID_ARG, "rtt_mcmc_sweep: measure_every must be >= 1");
    if (B == 0 || n_sweeps == 0) return RTT_OK;
    if (!spins || !state) return fail(RTT_ERR_INVALID_ARG, "rtt_mcmc_sweep: null spins or state");
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaGetLastError(), "rtt_mcmc_sweep: pending error");
    if ((s = ensure_scratch(h, B)) != RTT_OK) return s;
    const SimtArgs a = simt_args(h);
    auto sweeps = [&](int64_t sw0, int32_t n) -> rtt_status {
        if (n <= 0) return RTT_OK;
        if (h->precision >= RTT_BF16X3) {
            return tc_sweep(h, spins, state, B, chain0, sw0, n, n_accept, st);
        }
        prof_begin(h, KID_SWEEP, st);
        API_CUDA(h->precision == RTT_FP64
                     ? simt_sweep_f64(a, spins, state, B, chain0, sw0, n, h->seed, h->d_sw_rstack,
                                      h->d_sw_rexp, nullptr, nullptr, n_accept, st)
                     : simt_sweep_f32(a, spins, state, B, chain0, sw0, n, h->seed, h->d_sw_rstack,
                                      h->d_sw_rexp, nullptr, nullptr, n_accept, st),
                 "rtt_mcmc_sweep: sweep kernel");
        prof_end(h, KID_SWEEP, st);
        return RTT_OK;
    };
    if (!e_loc_trace) return sweeps(sweep0, n_sweeps);
    // Measured group g: the local energy of the configuration entering the
    // group runs on the handle's second stream, from a snapshot of the spins,
    // while the group's sweeps run on `stream`; the sweeps keep their own
    // environment stacks.  A snapshot buffer is reused two groups later, after
    // the energy that read it has finished; `stream` waits for the last energy
    // before the call's work ends.
    const int32_t n_meas = n_sweeps / measure_every;
    const size_t snap_bytes = (size_t)B * h->N;
    int64_t sw = sweep0;
    for (int32_t g = 0; g < n_meas; ++g) {
        uint8_t *snap = h->d_snap[g & 1];
        if (g >= 2) API_CUDA(cudaStreamWaitEvent(st, h->ev_done[g & 1], 0), "rtt_mcmc_sweep: wait");
        API_CUDA(cudaMemcpyAsync(snap, spins, snap_bytes, cudaMemcpyDeviceToDevice, st),
                 "rtt_mcmc_sweep: spin snapshot");
        API_CUDA(cudaEventRecord(h->ev_fork, st), "rtt_mcmc_sweep: fork");
        API_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0), "rtt_mcmc_sweep: fork");
        if ((s = energy_pipeline(h, snap, B, e_loc_trace + (size_t)g * B, nullptr, false,
                                 h->side)) != RTT_OK)
            return s;
        API_CUDA(cudaEventRecord(h->ev_done[g & 1], h->side), "rtt_mcmc_sweep: join");
        if ((s = sweeps(sw, measure_every)) != RTT_OK) return s;
        sw += measure_every;
    }
    if (n_meas > 0)
        API_CUDA(cudaStreamWaitEvent(st, h->ev_done[(n_meas - 1) & 1], 0), "rtt_mcmc_sweep: join");
    return sweeps(sw, n_sweeps - n_meas * measure_every);
}

rtt_status rtt_observables(rtt_handle h, const double *x, int32_t T, int64_t B,
                           const int64_t *n_accept, int64_t proposals_per_chain, rtt_stats *out,
                           void *stream) {
    g_last_error.clear();
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (!x || !out || T < 1 || B < 1)
        return fail(RTT_ERR_INVALID_ARG, "rtt_observables: need trace, out, T >= 1, B >= 1");
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaGetLastError(), "rtt_observables: pending error");
    const int chunk = 64;
    double *d_cm = nullptr, *d_acc = nullptr;
    unsigned long long *d_acc_i = nullptr;
    auto release = [&]() {
        cudaFree(d_cm);
        cudaFree(d_acc);
        cudaFree(d_acc_i);
    };
    auto cfail = [&](cudaError_t e, const char *w) {
        release();
        return cuda_fail(e, w);
    };
    cudaError_t e;
    if ((e = cudaMalloc((void **)&d_cm, (size_t)B * 8)) != cudaSuccess) return cfail(e, "stats alloc");
    if ((e = cudaMalloc((void **)&d_acc, (size_t)(chunk + 2) * 8)) != cudaSuccess)
        return cfail(e, "stats alloc");
    if ((e = cudaMalloc((void **)&d_acc_i, 8)) != cudaSuccess) return cfail(e, "stats alloc");
    if ((e = stats_chain_means(x, T, B, d_cm, st)) != cudaSuccess) return cfail(e, "chain means");
    std::vector<double> cm(B);
    if ((e = cudaMemcpyAsync(cm.data(), d_cm, (size_t)B * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cfail(e, "copy chain means");
    // lag sums in chunks until Sokal's window closes: W >= 5 tau(W)
    std::vector<double> rho;
    double c0 = 0.0, tau = 0.5;
    int W = 0;
    bool done = (T < 2);
    for (int lag0 = 0; lag0 < T && !done; lag0 += chunk) {
        const int nl = std::min(chunk, T - lag0);
        if ((e = cudaMemsetAsync(d_acc, 0, (size_t)nl * 8, st)) != cudaSuccess) return cfail(e, "memset");
        if ((e = stats_lag_sums(x, d_cm, T, B, lag0, nl, d_acc, st)) != cudaSuccess)
            return cfail(e, "lag sums");
        std::vector<double> acc(nl);
        if ((e = cudaMemcpyAsync(acc.data(), d_acc, (size_t)nl * 8, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return cfail(e, "copy lag sums");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cfail(e, "sync");
        for (int l = 0; l < nl && !done; ++l) {
            const int t = lag0 + l;
            const double ct = acc[l] / (double)B;
            if (t == 0) {
                c0 = ct;
                continue;
            }
            tau += (c0 > 0.0) ? ct / c0 : 0.0;
            W = t;
            if ((double)W >= 5.0 * tau) done = true;
        }
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cfail(e, "sync");
    tau = std::max(tau, 0.5);
    double mean = 0.0;
    for (int64_t c = 0; c < B; ++c) mean += cm[c];
    mean /= (double)B;
    double between = 0.0;
    for (int64_t c = 0; c < B; ++c) between += (cm[c] - mean) * (cm[c] - mean);
    // law of total variance over equal-length chains: within (C(0)) + between
    const double var = c0 + between / (double)B;
    const double n = (double)T * (double)B;
    rtt_stats r;
    memset(&r, 0, sizeof(r));
    r.mean = mean;
    r.var = var;
    r.tau_int = tau;
    r.window = W;
    r.ess = n / (2.0 * tau);
    r.se = sqrt(var * 2.0 * tau / n);
    r.n = (int64_t)n;
    r.v_score = mean != 0.0 ? (double)h->N * var / (mean * mean) : INFINITY;
    r.se_chain = (B >= 2) ? sqrt(between / (double)(B - 1)) / sqrt((double)B) : NAN;
    const int lb = (int)std::min<double>((double)T, std::max(1.0, ceil(20.0 * tau)));
    const int nb = T / lb;
    r.se_bin = NAN;
    if (nb >= 1 && (int64_t)nb * B >= 2) {
        if ((e = cudaMemsetAsync(d_acc, 0, 16, st)) != cudaSuccess) return cfail(e, "memset");
        if ((e = stats_bin_moments(x, T, B, lb, mean, d_acc, st)) != cudaSuccess)
            return cfail(e, "bin moments");
        double mo[2];
        if ((e = cudaMemcpyAsync(mo, d_acc, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cfail(e, "copy bins");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cfail(e, "sync");
        const double m = (double)nb * (double)B;
        const double vb = (mo[1] - mo[0] * mo[0] / m) / (m - 1.0);
        r.se_bin = sqrt(std::max(vb, 0.0) / m);
    }
    r.accept_rate = NAN;
    if (n_accept && proposals_per_chain > 0) {
        if ((e = cudaMemsetAsync(d_acc_i, 0, 8, st)) != cudaSuccess) return cfail(e, "memset");
        if ((e = stats_sum_i64(n_accept, B, d_acc_i, st)) != cudaSuccess) return cfail(e, "accepts");
        unsigned long long tot = 0;
        if ((e = cudaMemcpyAsync(&tot, d_acc_i, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cfail(e, "copy accepts");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cfail(e, "sync");
        r.accept_rate = (double)tot / ((double)B * (double)proposals_per_chain);
    }
    release();
    *out = r;
    return RTT_OK;
}

rtt_status rtt_profile(rtt_handle h, int32_t enable) {
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    DeviceGuard guard(h->device);
    API_CUDA(cudaDeviceSynchronize(), "rtt_profile: sync");
    Profiler *p = prof_of(h);
    p->reset();
    p->on = enable != 0;
    return RTT_OK;
}

rtt_status rtt_profile_read(rtt_handle h, rtt_kernel_time *out, int32_t capacity, int32_t *count) {
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (!count || capacity < 0 || (capacity > 0 && !out))
        return fail(RTT_ERR_INVALID_ARG, "rtt_profile_read: bad arguments");
    DeviceGuard guard(h->device);
    API_CUDA(cudaDeviceSynchronize(), "rtt_profile_read: sync");
    Profiler *p = prof_of(h);
    for (auto &r : p->pending) {
        float ms = 0.f;
        API_CUDA(cudaEventElapsedTime(&ms, r.a, r.b), "rtt_profile_read: elapsed");
        p->ms[r.kid] += ms;
        p->n[r.kid] += 1;
    }
    int32_t c = 0;
    for (int k = 0; k < KID_COUNT; ++k) {
        if (!p->n[k]) continue;
        if (c < capacity) out[c] = rtt_kernel_time{kKernelNames[k], p->n[k], p->ms[k]};
        ++c;
    }
    *count = c;
    const bool on = p->on;
    p->reset();
    p->on = on;
    return RTT_OK;
}

rtt_status rtt_device_status(rtt_handle h, int32_t *flags) {
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (!flags) return fail(RTT_ERR_INVALID_ARG, "rtt_device_status: null flags");
    DeviceGuard guard(h->device);
    API_CUDA(cudaDeviceSynchronize(), "rtt_device_status: sync");
    *flags = 0;
    int *w = tc_error_word(h);
    if (w) {
        int v = 0;
        API_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost), "rtt_device_status: read");
        API_CUDA(cudaMemset(w, 0, sizeof(int)), "rtt_device_status: clear");
        *flags = v;
    }
    if (*flags & 1) return fail(RTT_ERR_TIMEOUT, "a bounded device wait expired");
    return RTT_OK;
}

rtt_status rtt_wait_selftest(rtt_handle h, int64_t budget_cycles, void *stream) {
    rtt_status s = check_handle(h);
    if (s != RTT_OK) return s;
    if (!h->tc)
        return fail(RTT_ERR_UNSUPPORTED, "rtt_wait_selftest: needs a BF16X3 / FP16X3 handle");
    if (budget_cycles < 1000 || budget_cycles > 4000000000LL)
        return fail(RTT_ERR_INVALID_ARG, "rtt_wait_selftest: budget outside [1e3, 4e9] cycles");
    DeviceGuard guard(h->device);
    return tc_wait_selftest(h, (long long)budget_cycles, (cudaStream_t)stream);
}

rtt_status rtt_mcmc_uniforms(uint64_t seed, int64_t n, const uint64_t *counters, double *out,
                             void *stream) {
    g_last_error.clear();
    if (n < 0 || (n > 0 && (!counters || !out)))
        return fail(RTT_ERR_INVALID_ARG, "rtt_mcmc_uniforms: bad arguments");
    if (n == 0) return RTT_OK;
    API_CUDA(launch_uniforms(seed, n, counters, out, (cudaStream_t)stream), "rtt_mcmc_uniforms");
    return RTT_OK;
}

}  // extern "C"
