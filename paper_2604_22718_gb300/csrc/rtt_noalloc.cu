// rtt_noalloc.cu -- local energy that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a
// local-energy evaluation: real-time or embedded loops that forbid allocator
// calls after start-up, and programs whose device memory is handed out by an
// external pool manager that must own every allocation (a cudaMalloc behind
// its back would break its accounting or fail against its reservation).
// rtt_local_energy_noalloc serves them: it launches the
// same kernels as rtt_local_energy (left and right environments, flip rows,
// reduction), but their scratch comes from one fixed array compiled into the
// library instead of the handle's on-demand scratch, so the call itself
// performs no allocation.
//
// The array is a file-scope device global: every GPU that loads the library
// holds it (RTT_NOALLOC_SCRATCH_BYTES) until the process exits.  All calls
// share it and it keeps the previous call's contents; nothing needs clearing,
// because every scratch entry is written before it is read.  Calls that
// overlap on the GPU (two streams, or two threads without ordering) race on
// the array and corrupt each other's results.
#include <mutex>
#include <string>

#include "rtt_internal.cuh"

#define RTT_NOALLOC_SCRATCH_BYTES (32u << 20)
#define RTT_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[RTT_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[RTT_NOALLOC_MAX_DEVICES] = {nullptr};

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoallocLayout {
    size_t lstack, lexp, rstack, rexp, rows_mant, rows_exp, total;
};

NoallocLayout layout_for(const rtt_s *h, int64_t B) {
    const size_t eb = h->elem_bytes();
    const size_t nv = (size_t)B * h->N;
    NoallocLayout L;
    size_t off = 0;
    L.lstack = off;
    off += round256(nv * h->chip * eb);
    L.lexp = off;
    off += round256(nv * 4);
    L.rstack = off;
    off += round256(nv * h->chip * eb);
    L.rexp = off;
    off += round256(nv * 4);
    L.rows_mant = off;
    off += round256((size_t)B * (h->N + 1) * 8);
    L.rows_exp = off;
    off += round256((size_t)B * (h->N + 1) * 8);
    L.total = off;
    return L;
}

// Device address of the static array on the current device, looked up once
// per device with that device current.
cudaError_t scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

rtt_status noalloc_fail(rtt_status s, const std::string &msg) {
    rtt_set_error(msg);
    return s;
}

rtt_status noalloc_cuda(cudaError_t e, const char *where) {
    return noalloc_fail(RTT_ERR_CUDA, std::string("rtt_local_energy_noalloc: ") + where + ": " +
                                          cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

}  // namespace

extern "C" rtt_status rtt_local_energy_noalloc(rtt_handle h, const uint8_t *spins, int64_t B,
                                               double *e_loc, double *ratios, void *stream) {
    rtt_set_error("");
    if (!h) return noalloc_fail(RTT_ERR_INVALID_ARG, "rtt_local_energy_noalloc: null handle");
    if (B < 0) return noalloc_fail(RTT_ERR_INVALID_ARG, "rtt_local_energy_noalloc: B < 0");
    if (B == 0) return RTT_OK;
    if (!spins || !e_loc)
        return noalloc_fail(RTT_ERR_INVALID_ARG, "rtt_local_energy_noalloc: null spins or e_loc");
    if (h->precision != RTT_FP64 && h->precision != RTT_FP32)
        return noalloc_fail(RTT_ERR_UNSUPPORTED,
                            "rtt_local_energy_noalloc: only FP64 and FP32 handles are supported");
    if (!h->periodic)
        return noalloc_fail(RTT_ERR_UNSUPPORTED,
                            "rtt_local_energy_noalloc: only periodic paths are supported");
    // scratch bytes per chain before rounding: two stacks of N chi_p values,
    // their int32 exponents, and the rows' mantissas and exponents; a batch
    // beyond the area is rejected before any size is multiplied out, so no
    // product below can wrap around
    const size_t per_chain = (size_t)2 * h->N * h->chip * h->elem_bytes() + (size_t)8 * h->N +
                             (size_t)16 * (h->N + 1);
    if ((uint64_t)B > RTT_NOALLOC_SCRATCH_BYTES / per_chain)
        return noalloc_fail(RTT_ERR_INVALID_ARG,
                            "rtt_local_energy_noalloc: B = " + std::to_string(B) + " needs at least " +
                                std::to_string(per_chain) + " bytes of scratch per chain; the "
                                "static area holds " + std::to_string(RTT_NOALLOC_SCRATCH_BYTES) +
                                " bytes; split the batch");
    const NoallocLayout lay = layout_for(h, B);
    if (lay.total > RTT_NOALLOC_SCRATCH_BYTES) {
        const NoallocLayout one = layout_for(h, 1);
        const int64_t bmax = (int64_t)(RTT_NOALLOC_SCRATCH_BYTES / (one.total > 0 ? one.total : 1));
        return noalloc_fail(RTT_ERR_INVALID_ARG,
                            "rtt_local_energy_noalloc: B = " + std::to_string(B) + " needs " +
                                std::to_string(lay.total) + " bytes of scratch; the static area "
                                "holds " + std::to_string(RTT_NOALLOC_SCRATCH_BYTES) +
                                " bytes (about " + std::to_string(bmax) +
                                " chains for this handle); split the batch");
    }
    if (h->device < 0 || h->device >= RTT_NOALLOC_MAX_DEVICES)
        return noalloc_fail(RTT_ERR_UNSUPPORTED, "rtt_local_energy_noalloc: device ordinal >= 64");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return noalloc_cuda(e, "cudaGetDevice");
    const bool switch_dev = prev != h->device;
    if (switch_dev && (e = cudaSetDevice(h->device)) != cudaSuccess)
        return noalloc_cuda(e, "cudaSetDevice");
    rtt_status result = RTT_OK;
    void *base = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    do {
        if ((e = scratch_address(h->device, &base)) != cudaSuccess) {
            result = noalloc_cuda(e, "cudaGetSymbolAddress");
            break;
        }
        unsigned char *b = (unsigned char *)base;
        void *lstack = b + lay.lstack, *rstack = b + lay.rstack;
        int32_t *lexp = (int32_t *)(b + lay.lexp), *rexp = (int32_t *)(b + lay.rexp);
        double *rows_mant = (double *)(b + lay.rows_mant);
        int64_t *rows_exp = (int64_t *)(b + lay.rows_exp);
        const SimtArgs a{h->d_A, h->d_AT, h->d_bl, h->d_br, h->d_q, h->N, h->L, h->R, h->chip};
        const bool f64 = h->precision == RTT_FP64;
        e = f64 ? simt_left_env_f64(a, spins, B, lstack, lexp, st)
                : simt_left_env_f32(a, spins, B, lstack, lexp, st);
        if (e != cudaSuccess) { result = noalloc_cuda(e, "left environments"); break; }
        e = f64 ? simt_right_env_f64(a, spins, B, rstack, rexp, st)
                : simt_right_env_f32(a, spins, B, rstack, rexp, st);
        if (e != cudaSuccess) { result = noalloc_cuda(e, "right environments"); break; }
        e = f64 ? simt_rows_f64(a, spins, B, lstack, lexp, rstack, rexp, rows_mant, rows_exp, st)
                : simt_rows_f32(a, spins, B, lstack, lexp, rstack, rexp, rows_mant, rows_exp, st);
        if (e != cudaSuccess) { result = noalloc_cuda(e, "flip rows"); break; }
        e = eloc_reduce(spins, B, h->N, h->d_pos, h->d_bonds, h->n_bonds, h->J, h->h, rows_mant,
                        rows_exp, e_loc, ratios, st);
        if (e != cudaSuccess) { result = noalloc_cuda(e, "reduction"); break; }
    } while (0);
    if (switch_dev) cudaSetDevice(prev);
    return result;
}
