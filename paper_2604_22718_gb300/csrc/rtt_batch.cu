// rtt_batch.cu -- many RTT instances of uneven N, R and chi in one persistent
// launch (FP32 site contractions).
//
// One Monte Carlo iteration (one systematic sweep, Sec. 3.3, then the local
// energy of the new state, Sec. 3.3 / Sec. 4 Eq. ising-model) of every chain
// of every instance runs as ONE persistent kernel.  Work items are blocks of
// chains of one instance; they are sorted by estimated cost, longest first,
// and handed out by an atomic ticket counter, so instances whose per-chain
// work differs by four orders of magnitude share the GPU without a tail.
// An item runs the whole iteration for its chains (sweep, right environment,
// the N+1 flip rows, the reduction): there is no dependency between CTAs.
// The per-row arithmetic is the SIMT FP32 row of rtt_simt.cuh in the same
// order, so every instance reproduces its single-instance FP32 result bit for
// bit whatever the tile shape.
//
// Tile shape per (chi, L) bucket -- lanes per row and chains per item -- is
// chosen by a host-side autotuner (rtt_batch_tune) that times the candidates
// on the device and caches its choice in a small JSON file.  The launch is a
// node of an explicitly built CUDA graph whose parameters are updated per step.
#include <math.h>
#include <math_constants.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "rtt_simt.cuh"

struct BInst {
    const float *A, *AT, *bl, *br;
    const int32_t *q, *pos, *bonds;
    float *lstack, *rstack;
    int32_t *lexp, *rexp;
    int64_t spin_off, chain_off, B;
    double J, h;
    uint64_t seed;
    int N, L, R, chip, n_bonds, G, pad;
};

struct BItem {
    int inst;
    int count;
    int64_t begin;
};

struct rtt_batch_s {
    int device = 0;
    int n = 0;
    std::vector<rtt_handle> h;
    std::vector<char> tc;        // instance on the tensor cores (its own handle's sweep)
    std::vector<int64_t> B, chain_off, spin_off;
    int64_t total_chains = 0, total_spins = 0;
    std::vector<int> G, mult;    // per instance tile shape
    BInst *d_inst = nullptr;
    BItem *d_items = nullptr;
    int n_items = 0;
    size_t smem = 0;
    unsigned long long *d_counter = nullptr;
    unsigned long long base = 0;
    int grid = 0;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    void *g_spins = nullptr, *g_state = nullptr, *g_eloc = nullptr, *g_acc = nullptr;
};

namespace bt {

constexpr int NTB = 256;
constexpr unsigned FULL = 0xffffffffu;

struct StepArgs {
    const BInst *insts;
    const BItem *items;
    int n_items;
    unsigned long long *counter;
    unsigned long long base;
    uint8_t *spins;
    rtt_chain_state *state;
    int64_t sweep;
    double *e_loc;
    int64_t *n_accept;
    int n_max;
};

// One full iteration for one chain, by one group of GG lanes.
template <int CHI, int GG>
__device__ void iterate_chain(const BInst &I, int64_t cl, bool active, uint8_t *s, double *ratio,
                              const StepArgs &p, int gl) {
    using O = rttd::RowOps<float, CHI, GG>;
    rttd::KArgs a{I.A, I.AT, I.bl, I.br, I.q, I.N, I.L, I.R};
    const int N = I.N;
    const int64_t cg = I.chain_off + cl;  // global chain slot
    uint8_t *gsp = p.spins + I.spin_off + cl * N;
    for (int i = gl; i < N; i += GG) s[i] = gsp[i];
    __syncwarp();
    const float *A = I.A;
    float *rst = I.rstack + (size_t)cl * N * CHI;
    int32_t *rex = I.rexp + (size_t)cl * N;
    float *lst = I.lstack + (size_t)cl * N * CHI;
    int32_t *lex = I.lexp + (size_t)cl * N;
    double pm = p.state[cg].mant;
    int64_t pe = p.state[cg].exp2;
    int64_t acc_count = 0;
    const int span = (I.R - 1) * N;
    // ---- local energy of the configuration entering the sweep (as k_left_env,
    // k_right_env, k_rows, k_eloc_reduce); the sweep reuses the right environments
    rttd::right_env_chain<float, CHI, GG>(a, s, rst, rex, active, gl);
    {
        float u[O::NQ];
        O::load(I.bl, u, gl);
        int32_t E = 0;
        for (int j = 0; j < N; ++j) {
            O::vecmat(rttd::site<float, CHI>(A, j, s[__ldg(I.q + j)]), u, u, gl);
            E += O::renorm(u);
            if (active) {
                O::store(lst + (size_t)j * CHI, u, gl);
                if (gl == 0) lex[j] = E;
            }
        }
    }
    __syncwarp();
    double m0 = 0.0;
    int64_t e0 = 0;
    for (int jr = N; jr >= 0; --jr) {  // j = N first: psi(s) is the divisor
        const int j = jr;
        float u[O::NQ];
        int64_t E;
        if (j == 0) {
            O::load(I.bl, u, gl);
            E = 0;
        } else {
            O::load(lst + (size_t)(j - 1) * CHI, u, gl);
            E = lex[j - 1];
        }
        const int end = (j < N) ? (I.R - 1) * N + j : I.L - 1;
        int t = j % N;
        for (int k = j; k <= end; ++k) {
            const int sp = s[__ldg(I.q + t)] ^ ((t == j) ? 1 : 0);
            O::vecmat(rttd::site<float, CHI>(A, k, sp), u, u, gl);
            E += O::renorm(u);
            if (++t == N) t = 0;
        }
        const int rq = (j < N) ? j : N - 1;
        float r[O::NQ];
        O::load(rst + (size_t)rq * CHI, r, gl);
        E += rex[rq];
        double m = O::dot(u, r);
        rttd::normalize_scalar(m, E);
        if (j == N) {
            m0 = m;
            e0 = E;
        } else if (gl == 0) {
            ratio[__ldg(I.q + j)] = ldexp(m / m0, (int)(E - e0));
        }
    }
    __syncwarp();
    if (active && gl == 0) {
        double el;
        if (m0 == 0.0 || !isfinite(m0)) {
            el = CUDART_NAN;
        } else {
            int64_t zz = 0;
            for (int b = 0; b < I.n_bonds; ++b) {
                const int zi = 1 - 2 * (int)s[I.bonds[2 * b]];
                const int zj = 1 - 2 * (int)s[I.bonds[2 * b + 1]];
                zz += zi * zj;
            }
            double sum = 0.0;
            for (int i = 0; i < N; ++i) sum += ratio[i];
            el = I.J * (double)zz - I.h * sum;
        }
        p.e_loc[cg] = el;
    }
    __syncwarp();
    // ---- one sweep (as k_sweep), from the right environments above
    float l[O::NQ];
    O::load(I.bl, l, gl);
    int64_t El = 0;
    for (int j = 0; j < N; ++j) {
        const int i = __ldg(I.q + j);
        const int si = s[i];
        float u[O::NQ], keep[O::NQ];
        O::vecmat(rttd::site<float, CHI>(A, j, si ^ 1), l, u, gl);
        const int64_t Eu0 = El + O::renorm(u);
        O::vecmat(rttd::site<float, CHI>(A, j, si), l, keep, gl);
        const int64_t Ek = El + O::renorm(keep);
        float uf[O::NQ];
#pragma unroll
        for (int qq = 0; qq < O::NQ; ++qq) uf[qq] = u[qq];
        int64_t Eu = Eu0;
        int t = j + 1 == N ? 0 : j + 1;
        for (int k = j + 1; k <= j + span; ++k) {
            const int sp = s[__ldg(I.q + t)] ^ ((t == j) ? 1 : 0);
            O::vecmat(rttd::site<float, CHI>(A, k, sp), u, u, gl);
            Eu += O::renorm(u);
            if (++t == N) t = 0;
        }
        float r[O::NQ];
        O::load(rst + (size_t)j * CHI, r, gl);
        Eu += rex[j];
        double m = O::dot(u, r);
        rttd::normalize_scalar(m, Eu);
        const double rr = ldexp(m / pm, (int)(Eu - pe));
        const double x = rttd::mcmc_uniform(I.seed, (uint64_t)cl, (uint64_t)p.sweep, (uint64_t)j);
        const bool accept = x < rr * rr;
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
    __syncwarp();
    if (active && gl == 0) {
        p.state[cg].mant = pm;
        p.state[cg].exp2 = pe;
        if (p.n_accept) p.n_accept[cg] += acc_count;
    }
    __syncwarp();
    if (active)
        for (int i = gl; i < N; i += GG) gsp[i] = s[i];
    __syncwarp();
}

template <int CHI, int GG>
__device__ void run_item(const BInst &I, const BItem &it, const StepArgs &p, uint8_t *sm_sp,
                         double *sm_ratio) {
    constexpr int GROUPS = NTB / GG;
    const int grp = threadIdx.x / GG, gl = threadIdx.x % GG;
    uint8_t *s = sm_sp + (size_t)grp * p.n_max;
    double *ratio = sm_ratio + (size_t)grp * p.n_max;
    for (int base = 0; base < it.count; base += GROUPS) {
        const int off = base + grp;
        const bool active = off < it.count;
        const int64_t cl = it.begin + (active ? off : it.count - 1);
        iterate_chain<CHI, GG>(I, cl, active, s, ratio, p, gl);
    }
}

__global__ void __launch_bounds__(NTB, 1) k_batch(StepArgs p) {
    extern __shared__ unsigned char sm[];
    __shared__ int s_item;
    double *sm_ratio = (double *)sm;                      // [groups][n_max]
    uint8_t *sm_sp = sm + (size_t)(NTB / 16) * p.n_max * 8;  // [groups][n_max]
    while (true) {
        if (threadIdx.x == 0) {
            const unsigned long long t = atomicAdd(p.counter, 1ull);
            s_item = (t - p.base < (unsigned long long)p.n_items) ? (int)(t - p.base) : -1;
        }
        __syncthreads();
        const int it_idx = s_item;
        __syncthreads();
        if (it_idx < 0) break;
        const BItem it = p.items[it_idx];
        const BInst I = p.insts[it.inst];
        switch (I.chip * 100 + I.G) {
            case 3232: run_item<32, 32>(I, it, p, sm_sp, sm_ratio); break;
            case 3216: run_item<32, 16>(I, it, p, sm_sp, sm_ratio); break;
            case 6432: run_item<64, 32>(I, it, p, sm_sp, sm_ratio); break;
            case 6416: run_item<64, 16>(I, it, p, sm_sp, sm_ratio); break;
            case 12832: run_item<128, 32>(I, it, p, sm_sp, sm_ratio); break;
            case 12816: run_item<128, 16>(I, it, p, sm_sp, sm_ratio); break;
            case 25632: run_item<256, 32>(I, it, p, sm_sp, sm_ratio); break;
            default: break;
        }
        __syncthreads();
    }
}

}  // namespace bt

// ============================================================================ host
namespace {

rtt_status bfail(rtt_status s, const std::string &m) {
    rtt_set_error(m);
    return s;
}
rtt_status bcuda(cudaError_t e, const char *w) {
    return bfail(e == cudaErrorMemoryAllocation ? RTT_ERR_OOM : RTT_ERR_CUDA,
                 std::string(w) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

struct DevGuard {
    int prev = -1;
    bool changed = false;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) changed = cudaSetDevice(d) == cudaSuccess;
    }
    ~DevGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

int lbucket(int L) { return L <= 64 ? 0 : (L <= 256 ? 1 : 2); }

double chain_cost(const rtt_s *h) {
    const double span = (double)(h->R - 1) * h->N + 1;
    const double steps = 2.0 * h->N * span + (double)(h->R - 1) * h->N + 2.0 * h->N;
    return steps * (double)h->chip * h->chip;
}

bool valid_shape(int chip, int G) {
    if (G == 32) return chip >= 32;
    if (G == 16) return chip >= 32 && chip <= 128;
    return false;
}

// Build the item list (optionally restricted to a subset of instances and a
// cap on chains per instance) and upload it.
rtt_status build_items(rtt_batch_s *b, const std::vector<int> &which, int64_t cap_chains) {
    std::vector<std::pair<double, BItem>> items;
    for (int i : which) {
        const int groups = bt::NTB / b->G[i];
        const int per = groups * b->mult[i];
        const int64_t Bi = std::min<int64_t>(b->B[i], cap_chains);
        const double cost = chain_cost(b->h[i]) * per;
        for (int64_t c = 0; c < Bi; c += per) {
            BItem it;
            it.inst = i;
            it.begin = c;
            it.count = (int)std::min<int64_t>(per, Bi - c);
            items.push_back({cost, it});
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, BItem> &x, const std::pair<double, BItem> &y) {
                         return x.first > y.first;
                     });
    std::vector<BItem> flat;
    for (auto &p : items) flat.push_back(p.second);
    cudaFree(b->d_items);
    b->d_items = nullptr;
    b->n_items = (int)flat.size();
    if (flat.empty()) return RTT_OK;
    cudaError_t e = cudaMalloc((void **)&b->d_items, flat.size() * sizeof(BItem));
    if (e != cudaSuccess) return bcuda(e, "rtt_batch: items");
    e = cudaMemcpy(b->d_items, flat.data(), flat.size() * sizeof(BItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(e, "rtt_batch: items copy");
    return RTT_OK;
}

rtt_status upload_insts(rtt_batch_s *b) {
    std::vector<BInst> hi(b->n);
    for (int i = 0; i < b->n; ++i) {
        const rtt_s *h = b->h[i];
        BInst &I = hi[i];
        memset(&I, 0, sizeof(I));
        I.A = (const float *)h->d_A;
        I.AT = (const float *)h->d_AT;
        I.bl = (const float *)h->d_bl;
        I.br = (const float *)h->d_br;
        I.q = h->d_q;
        I.pos = h->d_pos;
        I.bonds = h->d_bonds;
        I.lstack = (float *)h->d_lstack;
        I.rstack = (float *)h->d_rstack;
        I.lexp = h->d_lexp;
        I.rexp = h->d_rexp;
        I.spin_off = b->spin_off[i];
        I.chain_off = b->chain_off[i];
        I.B = b->B[i];
        I.J = h->J;
        I.h = h->h;
        I.seed = h->seed;
        I.N = h->N;
        I.L = h->L;
        I.R = h->R;
        I.chip = h->chip;
        I.n_bonds = h->n_bonds;
        I.G = b->G[i];
    }
    if (!b->d_inst) {
        cudaError_t e = cudaMalloc((void **)&b->d_inst, hi.size() * sizeof(BInst));
        if (e != cudaSuccess) return bcuda(e, "rtt_batch: descriptors");
    }
    cudaError_t e = cudaMemcpy(b->d_inst, hi.data(), hi.size() * sizeof(BInst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(e, "rtt_batch: descriptors copy");
    return RTT_OK;
}

void drop_graph(rtt_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->node = nullptr;
}

bt::StepArgs step_args(rtt_batch_s *b, uint8_t *spins, rtt_chain_state *state, int64_t sweep,
                       double *e_loc, int64_t *n_accept) {
    int nmax = 1;
    for (int i = 0; i < b->n; ++i) nmax = std::max(nmax, b->h[i]->N);
    bt::StepArgs p;
    p.insts = b->d_inst;
    p.items = b->d_items;
    p.n_items = b->n_items;
    p.counter = b->d_counter;
    p.base = b->base;
    p.spins = spins;
    p.state = state;
    p.sweep = sweep;
    p.e_loc = e_loc;
    p.n_accept = n_accept;
    p.n_max = nmax;
    return p;
}

size_t smem_for(int nmax) { return (size_t)(bt::NTB / 16) * nmax * 9; }

rtt_status direct_launch(rtt_batch_s *b, const bt::StepArgs &p, cudaStream_t st) {
    if (b->n_items == 0) return RTT_OK;
    bt::k_batch<<<b->grid, bt::NTB, b->smem, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(e, "rtt_batch: launch");
    b->base += (unsigned long long)b->n_items + (unsigned long long)b->grid;
    return RTT_OK;
}

}  // namespace

extern "C" {

rtt_status rtt_batch_create(const rtt_desc *descs, int32_t n, const int64_t *chains, rtt_batch *out) {
    if (!descs || !chains || !out || n < 1)
        return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_create: need descs, chains, out and n >= 1");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (descs[i].precision != RTT_FP32 && descs[i].precision != RTT_FP16X3 &&
            descs[i].precision != RTT_BF16X3)
            return bfail(RTT_ERR_UNSUPPORTED, "rtt_batch_create: instances are FP32 (persistent "
                                              "kernel) or FP16X3 / BF16X3 (tensor cores)");
        if (descs[i].chi > 256 || chains[i] < 1)
            return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_create: chi <= 256 and chains >= 1 required");
        if (descs[i].device != descs[0].device)
            return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_create: all instances on one device");
    }
    rtt_batch_s *b = new rtt_batch_s();
    int dev = descs[0].device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete b;
        return bfail(RTT_ERR_CUDA, "rtt_batch_create: cudaGetDevice");
    }
    b->device = dev;
    DevGuard guard(dev);
    b->n = n;
    b->h.assign(n, nullptr);
    int nmax = 1;
    for (int i = 0; i < n; ++i) {
        rtt_desc d = descs[i];
        d.device = dev;
        rtt_status s = rtt_create(&d, &b->h[i]);
        if (s == RTT_OK && !b->h[i]->periodic)
            s = bfail(RTT_ERR_UNSUPPORTED, "rtt_batch_create: periodic paths only");
        const bool on_tc = d.precision != RTT_FP32;
        if (s == RTT_OK && !on_tc && b->h[i]->chip < 32) {
            rtt_destroy(b->h[i]);
            b->h[i] = nullptr;
            s = bfail(RTT_ERR_UNSUPPORTED, "rtt_batch_create: chi >= 17 required (32-lane rows)");
        }
        if (s == RTT_OK) s = rtt_reserve(b->h[i], chains[i]);
        if (s != RTT_OK) {
            rtt_batch_destroy(b);
            return s;
        }
        b->B.push_back(chains[i]);
        b->chain_off.push_back(b->total_chains);
        b->spin_off.push_back(b->total_spins);
        b->total_chains += chains[i];
        b->total_spins += chains[i] * b->h[i]->N;
        b->G.push_back(32);
        b->mult.push_back(1);
        b->tc.push_back(on_tc ? 1 : 0);
        if (!on_tc) nmax = std::max(nmax, b->h[i]->N);
    }
    cudaError_t e = cudaMalloc((void **)&b->d_counter, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        rtt_batch_destroy(b);
        return bcuda(e, "rtt_batch_create: counter");
    }
    cudaMemset(b->d_counter, 0, sizeof(unsigned long long));
    b->smem = smem_for(nmax);
    if (b->smem > 48 * 1024)
        cudaFuncSetAttribute(bt::k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bt::k_batch, bt::NTB, b->smem);
    b->grid = std::max(1, sms * std::max(per, 1));
    rtt_status s = upload_insts(b);
    std::vector<int> all;  // the persistent kernel's instances
    for (int i = 0; i < n; ++i)
        if (!b->tc[i]) all.push_back(i);
    if (s == RTT_OK) s = build_items(b, all, INT64_MAX);
    if (s != RTT_OK) {
        rtt_batch_destroy(b);
        return s;
    }
    *out = b;
    return RTT_OK;
}

rtt_status rtt_batch_destroy(rtt_batch b) {
    if (!b) return RTT_OK;
    {
        DevGuard guard(b->device);
        cudaDeviceSynchronize();
        drop_graph(b);
        cudaFree(b->d_inst);
        cudaFree(b->d_items);
        cudaFree(b->d_counter);
    }
    for (auto h : b->h)
        if (h) rtt_destroy(h);
    delete b;
    return RTT_OK;
}

rtt_status rtt_batch_layout(rtt_batch b, int64_t *total_chains, int64_t *total_spins,
                            int64_t *chain_off, int64_t *spin_off) {
    if (!b) return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_layout: null batch");
    if (total_chains) *total_chains = b->total_chains;
    if (total_spins) *total_spins = b->total_spins;
    for (int i = 0; i < b->n; ++i) {
        if (chain_off) chain_off[i] = b->chain_off[i];
        if (spin_off) spin_off[i] = b->spin_off[i];
    }
    return RTT_OK;
}

rtt_status rtt_batch_init(rtt_batch b, const uint8_t *spins, rtt_chain_state *state, void *stream) {
    if (!b || !spins || !state) return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_init: null argument");
    for (int i = 0; i < b->n; ++i) {
        rtt_status s = rtt_log_amplitudes(b->h[i], spins + b->spin_off[i], b->B[i], nullptr, nullptr,
                                          state + b->chain_off[i], stream);
        if (s != RTT_OK) return s;
    }
    return RTT_OK;
}

rtt_status rtt_batch_step(rtt_batch b, uint8_t *spins, rtt_chain_state *state, int64_t sweep,
                          double *e_loc, int64_t *n_accept, int32_t use_graph, void *stream) {
    if (!b || !spins || !state || !e_loc || sweep < 0)
        return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_step: null argument or negative sweep");
    DevGuard guard(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(e, "rtt_batch_step: pending error");
    // the tensor-core instances: one sweep of each on its own handle, measuring
    // the configuration it starts from (as the persistent kernel does), into
    // the instance's slices of the batch's arrays, after the persistent launch
    auto tc_steps = [&]() -> rtt_status {
        for (int i = 0; i < b->n; ++i) {
            if (!b->tc[i]) continue;
            rtt_status s = rtt_mcmc_sweep(b->h[i], spins + b->spin_off[i], state + b->chain_off[i],
                                          b->B[i], 0, sweep, 1, 1, e_loc + b->chain_off[i],
                                          n_accept ? n_accept + b->chain_off[i] : nullptr, stream);
            if (s != RTT_OK) return s;
        }
        return RTT_OK;
    };
    bt::StepArgs p = step_args(b, spins, state, sweep, e_loc, n_accept);
    if (!use_graph || b->n_items == 0) {
        rtt_status s = direct_launch(b, p, st);
        return s == RTT_OK ? tc_steps() : s;
    }
    if (b->exec && (b->g_spins != spins || b->g_state != state || b->g_eloc != e_loc ||
                    b->g_acc != (void *)n_accept))
        drop_graph(b);
    void *args[] = {&p};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void *)bt::k_batch;
    kp.gridDim = dim3(b->grid);
    kp.blockDim = dim3(bt::NTB);
    kp.sharedMemBytes = (unsigned)b->smem;
    kp.kernelParams = args;
    if (!b->exec) {
        if ((e = cudaGraphCreate(&b->graph, 0)) != cudaSuccess) return bcuda(e, "graph create");
        if ((e = cudaGraphAddKernelNode(&b->node, b->graph, nullptr, 0, &kp)) != cudaSuccess)
            return bcuda(e, "graph kernel node");
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
            return bcuda(e, "graph instantiate");
        b->g_spins = spins;
        b->g_state = state;
        b->g_eloc = e_loc;
        b->g_acc = n_accept;
    } else if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->node, &kp)) != cudaSuccess) {
        return bcuda(e, "graph node update");
    }
    if ((e = cudaGraphLaunch(b->exec, st)) != cudaSuccess) return bcuda(e, "graph launch");
    b->base += (unsigned long long)b->n_items + (unsigned long long)b->grid;
    return tc_steps();
}

// Autotuner: per (chi, L) bucket, time each candidate tile shape (lanes per
// row G, chains per item = groups * mult) on up to `probe_chains` chains of
// every instance in the bucket and keep the fastest per chain.  With a cache
// path, buckets found in the file are not re-timed and the file is rewritten
// with every bucket's choice.  SYNCHRONOUS.
rtt_status rtt_batch_tune(rtt_batch b, const char *cache_path, int32_t probe_chains, void *stream) {
    if (!b) return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_tune: null batch");
    if (probe_chains < 1) probe_chains = 64;
    DevGuard guard(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::map<std::pair<int, int>, std::vector<int>> buckets;
    for (int i = 0; i < b->n; ++i)
        if (!b->tc[i]) buckets[{b->h[i]->chip, lbucket(b->h[i]->L)}].push_back(i);
    std::map<std::pair<int, int>, std::pair<int, int>> chosen;  // -> (G, mult)
    std::map<std::pair<int, int>, double> best_ms;
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[256];
            while (fgets(line, sizeof(line), f)) {
                int chip, lb, G, mult;
                double ms;
                if (sscanf(line, " {\"chi\": %d, \"lbucket\": %d, \"G\": %d, \"mult\": %d, \"ms_per_chain\": %lf",
                           &chip, &lb, &G, &mult, &ms) == 5 && valid_shape(chip, G) && mult >= 1 && mult <= 8) {
                    chosen[{chip, lb}] = {G, mult};
                    best_ms[{chip, lb}] = ms;
                }
            }
            fclose(f);
        }
    }
    // scratch buffers for probing (device, own; freed before return)
    int64_t nch = 0, nsp = 0;
    for (int i = 0; i < b->n; ++i) {
        nch += b->B[i];
        nsp += b->B[i] * b->h[i]->N;
    }
    uint8_t *d_sp = nullptr;
    rtt_chain_state *d_st = nullptr;
    double *d_el = nullptr;
    cudaError_t e;
    auto release = [&]() {
        cudaFree(d_sp);
        cudaFree(d_st);
        cudaFree(d_el);
    };
    if ((e = cudaMalloc((void **)&d_sp, nsp)) != cudaSuccess) { release(); return bcuda(e, "tune"); }
    if ((e = cudaMalloc((void **)&d_st, nch * sizeof(rtt_chain_state))) != cudaSuccess) { release(); return bcuda(e, "tune"); }
    if ((e = cudaMalloc((void **)&d_el, nch * sizeof(double))) != cudaSuccess) { release(); return bcuda(e, "tune"); }
    cudaMemsetAsync(d_sp, 0, nsp, st);
    rtt_status s = rtt_batch_init(b, d_sp, d_st, st);
    if (s != RTT_OK) { release(); return s; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int Gs[2] = {32, 16};
    const int mults[2] = {1, 2};
    for (auto &kv : buckets) {
        if (chosen.count(kv.first)) {
            for (int i : kv.second) {
                b->G[i] = chosen[kv.first].first;
                b->mult[i] = chosen[kv.first].second;
            }
            continue;
        }
        double best = 1e300;
        std::pair<int, int> pick{32, 1};
        for (int G : Gs) {
            if (!valid_shape(kv.first.first, G)) continue;
            for (int mult : mults) {
                for (int i : kv.second) {
                    b->G[i] = G;
                    b->mult[i] = mult;
                }
                if ((s = upload_insts(b)) != RTT_OK) break;
                if ((s = build_items(b, kv.second, probe_chains)) != RTT_OK) break;
                int64_t probed = 0;
                for (int i : kv.second) probed += std::min<int64_t>(b->B[i], probe_chains);
                bt::StepArgs p = step_args(b, d_sp, d_st, 0, d_el, nullptr);
                cudaEventRecord(e0, st);
                s = direct_launch(b, p, st);
                cudaEventRecord(e1, st);
                if (s != RTT_OK) break;
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double per = ms / (double)std::max<int64_t>(probed, 1);
                if (per < best) {
                    best = per;
                    pick = {G, mult};
                }
            }
            if (s != RTT_OK) break;
        }
        if (s != RTT_OK) break;
        chosen[kv.first] = pick;
        best_ms[kv.first] = best;
        for (int i : kv.second) {
            b->G[i] = pick.first;
            b->mult[i] = pick.second;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    if (s != RTT_OK) return s;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bcuda(e, "tune sync");
    drop_graph(b);
    if ((s = upload_insts(b)) != RTT_OK) return s;
    std::vector<int> all;
    for (int i = 0; i < b->n; ++i)
        if (!b->tc[i]) all.push_back(i);
    if ((s = build_items(b, all, INT64_MAX)) != RTT_OK) return s;
    if (cache_path) {
        FILE *f = fopen(cache_path, "w");
        if (f) {
            fprintf(f, "{\"tile_shapes\": [\n");
            size_t k = 0;
            for (auto &kv : chosen) {
                fprintf(f, "  {\"chi\": %d, \"lbucket\": %d, \"G\": %d, \"mult\": %d, \"ms_per_chain\": %.6g}%s\n",
                        kv.first.first, kv.first.second, kv.second.first, kv.second.second,
                        best_ms[kv.first], (++k < chosen.size()) ? "," : "");
            }
            fprintf(f, "]}\n");
            fclose(f);
        }
    }
    return RTT_OK;
}

rtt_status rtt_batch_shape(rtt_batch b, int32_t instance, int32_t *lanes, int32_t *chains_per_item) {
    if (!b || instance < 0 || instance >= b->n)
        return bfail(RTT_ERR_INVALID_ARG, "rtt_batch_shape: bad instance");
    if (lanes) *lanes = b->G[instance];
    if (chains_per_item) *chains_per_item = (bt::NTB / b->G[instance]) * b->mult[instance];
    return RTT_OK;
}

}  // extern "C"
