// rtt_tc.cu -- tensor-core form of the RTT site chain (sm_103a, tcgen05).
//
// Per site k the rows of a 128-chain tile are multiplied by the slice of
// their own spin, v <- v A_k[s] (Eq. RTT evaluated left to right; right-to-
// left steps use the transposed slices), on the 5th-generation tensor cores:
//   - operands in 16-bit hi/lo split form, x = hi + lo + O(u^2 |x|) with u
//     the unit roundoff of the 16-bit type (BF16: 2^-8, FP16: 2^-11); three
//     products hi.hi + hi.lo + lo.hi accumulate in FP32 in TMEM.  Each site
//     tensor is prescaled by an exact power of two 2^c_k (max entry in [1,2))
//     so that FP16 stays in its normal range; c_k is taken back out of the
//     integer exponent sum;
//   - the two slices are interleaved along K, so a row's operand is 2:4
//     sparse and one tcgen05.mma.sp with a per-row metadata word computes
//     exactly the row's own slice (SCfg); the chi = 64 split-row sweep keeps
//     the dense form, both slices at once (N = 2 chi) and a per-row select;
//   - the site tensors are streamed by TMA (128-byte swizzle, K-major) into a
//     ring of shared-memory stages; the rows live in tensor memory as the A
//     operand, written by the epilogue;
//   - epilogue: load the accumulator, rescale by an exact power of two
//     (exponent summed in an integer), split to hi/lo and store the row back
//     as the next site's A operand, with the next site's metadata.
// A producer warp issues TMA and MMA; every wait is bounded by a clock budget
// after which the CTA records an error flag, drains its own copies, frees
// its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rtt_internal.cuh"
#include "rtt_tcgen05.cuh"

struct TcPlan {
    int chi = 0;
    bool f16 = false;              // FP16 operands (else BF16)
    // dense operand (chi = 64 split-row sweep): [4][L][2chi][chi], rows = output
    // (s, b) of the left-to-right form (planes 0 hi, 1 lo) or (s, a) of the
    // right-to-left form (planes 2, 3), K = the contracted index
    uint16_t *d_B = nullptr;
    CUtensorMap map;
    // sparse operand (k_tc): [4][L][chi][2chi], rows = output b (planes 0, 1)
    // or a (planes 2, 3), K = 2 x + s over the contracted index x and slice s
    uint16_t *d_Bs = nullptr;
    CUtensorMap map_sp;
    int32_t *d_cexp = nullptr;     // [L] prescale exponents c_k
    float *d_bl = nullptr, *d_br = nullptr;
    float *d_tmp = nullptr;  // [B][chi] sweep scratch (flipped start of a row)
    int32_t *d_tmp_exp = nullptr;
    int64_t tmp_cap = 0;
    int *d_err = nullptr;    // device error flags (bit 0: a bounded wait expired)
};

bool tc_supported_chi(int chi) { return chi == 64 || chi == 128; }

namespace tcd {

constexpr int NT = 128;  // threads per CTA = rows per tile = TMEM lanes
constexpr int NS = 2;    // B-operand ring stages
constexpr unsigned FULL = 0xffffffffu;

enum { M_ROWS = 0, M_LEFT = 1, M_RIGHT = 2, M_INIT = 3, M_SWEEP = 4 };

template <int CHI, bool F16 = false>
struct Cfg {
    static constexpr int KA = CHI / 64;            // 64-element K atoms per row
    static constexpr int BOX = 2 * CHI * 128;      // bytes: 2chi rows x 128 B
    static constexpr int STAGE = 2 * BOX;          // hi box + lo box
    static constexpr int TCOLS = 2 * CHI;          // accumulator columns
    static constexpr int A_COL = 2 * CHI;          // row hi at A_COL, lo at A_COL + CHI/2
    static constexpr int TALLOC = 3 * CHI <= 256 ? 256 : 512;  // columns allocated
    // kind::f16, (BF16 or FP16) x same -> FP32, both K-major, N = 2chi, M = 128
    static constexpr uint32_t FMT = F16 ? 0u : 1u;
    static constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) |
                                      ((uint32_t)((2 * CHI) >> 3) << 17) |
                                      ((uint32_t)(128 >> 4) << 24);
    static constexpr int CTRL = 128;
    static size_t smem_bytes(int N, int L) {
        return 1024 + (size_t)NS * STAGE + CTRL + (size_t)16 * N + (size_t)4 * L;
    }
};

// The sparse form of a site product (generic tile kernel k_tc).  A row needs
// only the slice of its spin, so the two slices are interleaved along K
// (K index 2a + s, K = 2chi) and the row operand is 2:4 sparse: in every
// group of four K entries (a, a+1 with both slices) the row keeps the two of
// its slice.  tcgen05.mma.sp reads the row's chi values as the compressed
// operand and a per-row metadata word that names the kept positions of each
// group -- (0,2) for slice 0, (1,3) for slice 1 -- and runs at twice the dense
// rate: one MMA of N = chi, logical K = 32 per 16 row entries, and the
// accumulator holds exactly the selected product (no discarded half).
//
// Metadata in tensor memory (measured on GB300 with one-row-per-lane words
// that differ from lane to lane, M = 128, K = 32 per instruction): row m's
// 32-bit metadata (nibble g = group g: first kept position in bits 0-1,
// second in bits 2-3) is not lane m's column entry.  Within the row's 32-lane
// group, with i = m mod 32 = 16u + 8v + w, its low 16 bits are half v of
// lane 16u + w and its high 16 bits half v of lane 16u + 8 + w.  A slice
// word has equal halves (0x8888 | 0x8888 << 16 or 0xDDDD | 0xDDDD << 16), so
// lane l = 16u + 8t + w holds, in half v, the 16-bit pattern of row
// 16u + 8v + w -- assembled with two shuffles.  The metadata column address
// must be aligned: every column used here is a multiple of 64.
template <int CHI, bool F16 = false>
struct SCfg {
    // B-operand ring stages of one 64-element K atom (hi and lo boxes): each
    // atom's stage is refilled with the next site's atom as soon as the MMAs
    // that read it complete (six stages at chi = 128 measured slower)
    static constexpr int NSTG = 4;
    static constexpr int KA = 2 * CHI / 64;        // 64-element K atoms per site
    static constexpr int BOX = CHI * 128;          // bytes: chi rows x 128 B
    static constexpr int STAGE = 2 * BOX;          // hi box + lo box
    static constexpr int ACC2 = CHI;               // second accumulator (sweep: unflipped l_j)
    static constexpr int A_COL = 2 * CHI;          // row hi at A_COL, lo at A_COL + CHI/2
    static constexpr int META = 3 * CHI;           // metadata of ACC (a multiple of 64)
    static constexpr int META2 = META + 64;        // metadata of ACC2 (sweep only)
    // columns allocated: a power of two covering what the mode uses
    static constexpr uint32_t TALLOC = META + 1 <= 256 ? 256u : 512u;
    static constexpr uint32_t TALLOC_SWEEP = META2 + 1 <= 256 ? 256u : 512u;
    // kind::f16, 2:4 sparse A (bit 2, selector 0), (BF16 or FP16) x same ->
    // FP32, both K-major, N = chi, M = 128
    static constexpr uint32_t FMT = F16 ? 0u : 1u;
    static constexpr uint32_t IDESC = (1u << 2) | (1u << 4) | (FMT << 7) | (FMT << 10) |
                                      ((uint32_t)(CHI >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    static constexpr uint32_t HALF0 = 0x8888u;  // groups keep positions (0, 2): slice 0
    static constexpr uint32_t HALF1 = 0xDDDDu;  // positions (1, 3): slice 1
    static constexpr int CTRL = 128;
    // epilogue: NH warps per TMEM lane quadrant (one: with a separate producer
    // warp, two per quadrant would cap the registers below what the sweep
    // needs), each thread owning CPT 64-column chunks of its row; with NH = 2
    // the halves of a row exchange the row maximum (two kinds per site) and the
    // closing dot product
    static constexpr int NH = 1;
    static constexpr int CPT = CHI / 64 / NH;
    static constexpr int XCH = NH * 128 * (2 * 4 + 8);
    static size_t smem_bytes(int N, int L) {
        return 1024 + (size_t)NSTG * STAGE + CTRL + (size_t)16 * N + (size_t)4 * L + 16 + XCH;
    }
};

struct Args {
    const float *bl, *br;
    const int32_t *q;
    const int32_t *cexp;
    int N, L, R;
    int64_t B;
    const uint8_t *spins_in;
    uint8_t *spins_out;
    float *lstack;
    int32_t *lexp;
    float *rstack;
    int32_t *rexp;
    double *rows_mant;
    int64_t *rows_exp;
    double *log_abs;
    int8_t *sign;
    rtt_chain_state *state;
    float *tmp;
    int32_t *tmp_exp;
    // path: general paths give the spin of every site (nullptr: periodic,
    // site k carries q[k mod N]); last[i] is spin i's last site; the right
    // stacks hold r_{kmin+e} at entry e < nr (entry nr-1 = L - kmin is b_R)
    const int32_t *path;
    const int32_t *last;
    int kmin, nr;
    int64_t chain0, sweep0;
    int n_sweeps;
    uint64_t seed;
    int64_t *n_accept;
    int *err;
    long long wait_limit;
};

// PTX wrappers: rtt_tcgen05.cuh
// ------------------------------------------------------------------ row helpers
// ---- 64-column chunks of a row (the epilogue never holds a whole chi = 128
// row in registers)
__device__ __forceinline__ void tmem_ld_64(uint32_t t, float (&y)[64]) {
    uint32_t x0[32], x1[32];
    tmem_ld_2x32(t, t + 32, x0, x1);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        y[i] = __uint_as_float(x0[i]);
        y[32 + i] = __uint_as_float(x1[i]);
    }
}
// y <- y 2^-e (exact; e = 0 leaves y)
__device__ __forceinline__ void scale_chunk(float (&y)[64], int e) {
    if (e == 0) return;
    if (rttd::pow2_normal(0.f, -e)) {
        const float sc = rttd::pow2(0.f, -e);
#pragma unroll
        for (int i = 0; i < 64; ++i) y[i] *= sc;
    } else {
#pragma unroll
        for (int i = 0; i < 64; ++i) y[i] = rttd::scale2(y[i], -e);
    }
}
__device__ __forceinline__ void load_chunk(const float *__restrict__ p, float (&y)[64]) {
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float4 x = p4[i];
        y[4 * i] = x.x;
        y[4 * i + 1] = x.y;
        y[4 * i + 2] = x.z;
        y[4 * i + 3] = x.w;
    }
}
__device__ __forceinline__ void store_chunk(float *__restrict__ p, const float (&y)[64]) {
    float4 *p4 = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int i = 0; i < 16; ++i) p4[i] = make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
}
// Chunk c of the closing contraction sum_b v_b r_b into eight FP32 partial
// sums (r points at entry 64 c); dot_finish combines them in FP64.  The
// partial a term goes to depends only on its index, so the chunks add up in
// the order of one pass over the whole row.
__device__ __forceinline__ void dot_chunk(const float (&y)[64], const float *__restrict__ r,
                                          float (&acc)[8]) {
    const float4 *r4 = reinterpret_cast<const float4 *>(r);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float4 x = r4[i];
        const int p = (2 * i) & 7;
        acc[p] = fmaf(y[4 * i], x.x, acc[p]);
        acc[p + 1] = fmaf(y[4 * i + 1], x.y, acc[p + 1]);
        acc[(p + 2) & 7] = fmaf(y[4 * i + 2], x.z, acc[(p + 2) & 7]);
        acc[(p + 3) & 7] = fmaf(y[4 * i + 3], x.w, acc[(p + 3) & 7]);
    }
}
__device__ __forceinline__ double dot_finish(const float (&acc)[8]) {
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < 8; ++p) s += (double)acc[p];
    return s;
}

// One 32-bit column of this warp's 32 TMEM lanes, then wait.
__device__ __forceinline__ void tmem_st_1(uint32_t t, uint32_t x) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(t), "r"(x)
        : "memory");
}

// Split two entries into 16-bit hi/lo (x = hi + lo + O(u^2 |x|)).
template <bool F16>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &h, uint32_t &l) {
    if (F16) {
        const __half2 hb = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(hb);
        const __half2 lb = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
        h = *reinterpret_cast<const uint32_t *>(&hb);
        l = *reinterpret_cast<const uint32_t *>(&lb);
    } else {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        h = *reinterpret_cast<const uint32_t *>(&hb);
        l = *reinterpret_cast<const uint32_t *>(&lb);
    }
}

template <int CHI>
__device__ __forceinline__ void load_vec(const float *__restrict__ p, float (&v)[CHI]) {
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < CHI / 4; ++i) {
        const float4 x = p4[i];
        v[4 * i] = x.x;
        v[4 * i + 1] = x.y;
        v[4 * i + 2] = x.z;
        v[4 * i + 3] = x.w;
    }
}
template <int CHI>
__device__ __forceinline__ void store_vec(float *__restrict__ p, const float (&v)[CHI]) {
    float4 *p4 = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int i = 0; i < CHI / 4; ++i) p4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ void normalize_scalar(double &m, int64_t &e) {
    if (m == 0.0 || !isfinite(m)) return;
    const int k = rttd::exponent_of(m);
    m = rttd::scale2(m, -k);
    e += k;
}

// Store 32 columns at t0 and 32 at t1 of this warp's 32 TMEM lanes, then wait.
__device__ __forceinline__ void tmem_st_2x32(uint32_t t0, uint32_t t1, const uint32_t (&x)[32],
                                             const uint32_t (&y)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%1], {%34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63, %64, %65};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(t0), "r"(t1), "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]), "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), "r"(x[14]), "r"(x[15]), "r"(x[16]), "r"(x[17]), "r"(x[18]), "r"(x[19]), "r"(x[20]), "r"(x[21]), "r"(x[22]), "r"(x[23]), "r"(x[24]), "r"(x[25]), "r"(x[26]), "r"(x[27]), "r"(x[28]), "r"(x[29]), "r"(x[30]), "r"(x[31]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(y[7]), "r"(y[8]), "r"(y[9]), "r"(y[10]), "r"(y[11]), "r"(y[12]), "r"(y[13]), "r"(y[14]), "r"(y[15]), "r"(y[16]), "r"(y[17]), "r"(y[18]), "r"(y[19]), "r"(y[20]), "r"(y[21]), "r"(y[22]), "r"(y[23]), "r"(y[24]), "r"(y[25]), "r"(y[26]), "r"(y[27]), "r"(y[28]), "r"(y[29]), "r"(y[30]), "r"(y[31])
        : "memory");
}
// Chunk c (entries 64 c .. 64 c + 63) of the row as the A operand in TMEM,
// row m in lane m: the 16-bit hi/lo split, entries 2i and 2i+1 in one column
// (lower index in the low half), hi at t_hi + 32 c, lo at t_hi + CHI/2 + 32 c.
template <int CHI, bool F16>
__device__ __forceinline__ void write_A_chunk(uint32_t t_hi, int c, const float (&y)[64]) {
    uint32_t h[32], l[32];
#pragma unroll
    for (int p = 0; p < 32; ++p) split2<F16>(y[2 * p], y[2 * p + 1], h[p], l[p]);
    tmem_st_2x32(t_hi + (uint32_t)(32 * c), t_hi + (uint32_t)(CHI / 2 + 32 * c), h, l);
}

// D (+)= A . B with A read from TMEM (K-major rows in TMEM lanes) and B from a
// shared-memory descriptor.
__device__ __forceinline__ void mma_f16_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                           uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// D (+)= A . B with A 2:4 sparse: its compressed entries read from TMEM (row
// m in lane m), the positions they take from the per-lane metadata column at
// `meta`, B dense from a shared-memory descriptor.
__device__ __forceinline__ void mma_sp_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t meta,
                                          uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %5, 0;\n\t"
        "tcgen05.mma.sp.cta_group::1.kind::f16 [%0], [%1], %2, [%3], %4, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(meta), "r"(idesc), "r"(accum)
        : "memory");
}

// Named barrier over n threads (id 1..15; id 0 is __syncthreads).
__device__ __forceinline__ void bar_sync_n(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// ------------------------------------------------------------------ site program
// A cursor walks the sites a CTA visits, in order, without divisions:
//   ROWS   k = j, j+1, ...            (left to right)
//   LEFT   k = 0 .. N-1               INIT  k = 0 .. L-1
//   RIGHT  k = L-1 .. (R-1)N+1        (right to left)
//   SWEEP  per sweep: right environment (form 1, k = L-1 .. (R-1)N+1),
//          then for jj = 0..N-1 the flip row k = jj .. jj + (R-1)N (form 0)
struct Cursor {
    int k, form;  // form 0: left-to-right (BT planes), 1: right-to-left (B planes)
    int tt;       // sweep: right-environment step
    int jj, i;    // sweep: proposal and position in its row
    int sw;       // sweep number
};

template <int MODE>
__device__ __forceinline__ Cursor cursor_start(const Args &a, int j) {
    Cursor c{0, 0, 0, 0, 0, 0};
    if (MODE == M_ROWS) c.k = j;
    if (MODE == M_RIGHT) {
        c.k = a.L - 1;
        c.form = 1;
    }
    if (MODE == M_SWEEP && a.N > 1) {
        c.k = a.L - 1;
        c.form = 1;
    }
    return c;
}

template <int MODE>
__device__ __forceinline__ void cursor_next(Cursor &c, const Args &a, int span) {
    if (MODE == M_ROWS || MODE == M_LEFT || MODE == M_INIT) {
        ++c.k;
    } else if (MODE == M_RIGHT) {
        --c.k;
    } else if (c.form == 1) {
        ++c.tt;
        --c.k;
        if (c.tt == a.N - 1) {
            c.form = 0;
            c.jj = 0;
            c.i = 0;
            c.k = 0;
        }
    } else {
        ++c.i;
        ++c.k;
        if (c.i == span) {
            ++c.jj;
            c.i = 0;
            c.k = c.jj;
            if (c.jj == a.N) {
                ++c.sw;
                c.jj = 0;
                c.k = 0;
                c.tt = 0;
                if (a.N > 1) {
                    c.form = 1;
                    c.k = a.L - 1;
                }
            }
        }
    }
}

// Last site of flip row j (j < N flips the spin of site j; j = N is psi(s)).
__device__ __forceinline__ int row_end(const Args &a, int j) {
    if (j >= a.N) return a.L - 1;
    if (a.path) return __ldg(a.last + __ldg(a.path + j));
    return j + (a.R - 1) * a.N;
}

template <int MODE>
__device__ __forceinline__ long long n_steps_of(const Args &a, int j) {
    const int span = (a.R - 1) * a.N + 1;
    if (MODE == M_ROWS) return row_end(a, j) - j + 1;
    if (MODE == M_LEFT) return a.N;
    if (MODE == M_RIGHT) return a.L - a.kmin;
    if (MODE == M_INIT) return a.L;
    return (long long)a.n_sweeps * ((a.N - 1) + (long long)a.N * span);
}

// ------------------------------------------------------------------ kernel
// One 128-chain tile per CTA (row m = TMEM lane m).  A producer warp (lane 0)
// streams the site tensors by TMA into a ring of NSTG stages and issues the
// sparse MMAs of each site, refilling each stage while the epilogue of the
// site runs; the epilogue runs on NH = chi/64 warps per TMEM lane quadrant, warp
// (quadrant q, half h) owning rows 32q..32q+31 and columns [64h, 64h+64):
// each thread loads its 64 accumulator columns once, the two halves of a row
// agree on the row maximum (renormalisation) and, at a decision, on the
// closing dot product through shared memory (a 32 NH-thread named barrier
// per quadrant); then each scales its chunk, writes it into the next A
// operand and into the stacks.  The h = 0 warps keep the spin bits and write
// the next site's metadata.  In the sweep, the first site of a proposal row
// is contracted with both slices (two accumulators): the kept continuation
// l_j and the flipped start of the row.
template <int CHI, int MODE, bool F16>
__global__ void __launch_bounds__(NT * SCfg<CHI, F16>::NH + 32, 1)
    k_tc(const __grid_constant__ CUtensorMap map, const Args a) {
    using C = SCfg<CHI, F16>;
    constexpr int NSG = C::NSTG;
    constexpr int NH = C::NH;
    constexpr int CPT = C::CPT;
    constexpr int NTH = NT * NH + 32;  // epilogue warps and the producer warp
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t stage0 = sa(base);
    uint64_t *bars = (uint64_t *)(base + NSG * C::STAGE);
    const uint32_t bar0 = sa(bars);
    // bars: full[0..NSG), empty[0..NSG), mma_done
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (NSG + s); };
    const uint32_t done_bar = bar0 + 8u * (2 * NSG);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NSG + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    uint32_t *bits = (uint32_t *)(base + NSG * C::STAGE + C::CTRL);
    // site table: low 16 bits spin q[k mod N], high 16 bits the prescale c_k
    uint32_t *tab = bits + 4 * a.N;
    // exchange slots: row maxima [2 kinds][NH][128], dot products [NH][128]
    float *xmax = (float *)(((uintptr_t)(tab + a.L) + 15) & ~(uintptr_t)15);
    double *xdot = (double *)(xmax + 2 * NH * NT);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool epi = warp < 4 * NH;         // an epilogue warp (else the producer)
    const bool issuer = warp == 4 * NH && lane == 0;
    const int q = warp & 3, h = epi ? warp >> 2 : 0;  // TMEM lane quadrant, column half
    const int m = 32 * q + lane;            // row of the tile
    const int64_t c_raw = (int64_t)blockIdx.x * NT + m;
    const bool active = c_raw < a.B;
    const bool lead = epi && active && h == 0;  // the thread that writes the row's scalars
    const int64_t c = active ? c_raw : a.B - 1;
    const int j = (MODE == M_ROWS) ? (int)blockIdx.y : 0;
    const int N = a.N;
    const int span = (a.R - 1) * N + 1;
    const int rbase = a.kmin;  // first site the right stack holds
    const long long total_steps = n_steps_of<MODE>(a, j);
    const long long total_atoms = total_steps * C::KA;

    constexpr uint32_t TALLOC = MODE == M_SWEEP ? C::TALLOC_SWEEP : C::TALLOC;
    if (warp == 0) tmem_alloc(sa(tmem_slot), TALLOC);
    if (issuer) {
        for (int s = 0; s < NSG; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    for (int k = tid; k < a.L; k += NTH)
        tab[k] = ((uint32_t)__ldg(a.path ? a.path + k : a.q + (k % N)) & 0xffffu) |
                 ((uint32_t)(__ldg(a.cexp + k) & 0xffff) << 16);
    // spin bits: word (i, quadrant) holds bit (row & 31) = s_i of that row's chain
    if (epi && h == 0) {
        for (int i = 0; i < N; ++i) {
            const uint32_t w = __ballot_sync(FULL, a.spins_in[c * N + i] != 0);
            if (lane == 0) bits[i * 4 + q] = w;
        }
    }
    auto spin = [&](int i) -> int { return (int)((bits[i * 4 + q] >> lane) & 1u); };
    auto site_spin = [&](int k) -> int { return (int)(tab[k] & 0xffffu); };
    auto site_cexp = [&](int k) -> int { return (int)(int16_t)(tab[k] >> 16); };
    const int iflip = (MODE == M_ROWS && j < N) ? (int)(__ldg(a.path ? a.path + j : a.q + j)) : -1;
    // the slice this row takes at the site of cursor x (the flipped spin's
    // slice is the other one); in the sweep the first site of a row also
    // takes the kept slice, into the second accumulator
    auto slice_of = [&](const Cursor &x) -> int {
        const int sk = site_spin(x.k);
        if (MODE == M_ROWS) return spin(sk) ^ (sk == iflip ? 1 : 0);
        if (MODE == M_SWEEP && x.form == 0) return spin(sk) ^ (sk == site_spin(x.jj) ? 1 : 0);
        return spin(sk);
    };
    // the halves of a row agree on its maximum and on its closing dot product
    auto row_max = [&](float mx, int kind) -> float {
        if (NH == 1) return mx;
        xmax[(kind * NH + h) * NT + m] = mx;
        bar_sync_n(1 + q, 32 * NH);
        return fmaxf(mx, xmax[(kind * NH + (h ^ 1)) * NT + m]);
    };
    auto row_dot = [&](double s) -> double {
        if (NH == 1) return s;
        xdot[h * NT + m] = s;
        bar_sync_n(1 + q, 32 * NH);
        return xdot[m] + xdot[NT + m];
    };

    // start row: written straight into the A operand (and, for the right
    // environments, b_R as the stack's last entry)
    int64_t E = 0;      // exponent of the current row
    int64_t El = 0;     // sweep: exponent of l_{jj-1}
    int64_t Ekeep = 0, Eflip = 0;
    double pm = 0.0;
    int64_t pe = 0, acc_count = 0;
    double fin_m = 0.0;  // rows / amplitude: the closing contraction
    int64_t fin_E = 0;
    const float *start = a.bl;
    if (MODE == M_ROWS && j > 0) {
        start = a.lstack + ((size_t)c * N + (j - 1)) * CHI;
        E = a.lexp[(size_t)c * N + (j - 1)];
    } else if (MODE == M_RIGHT || MODE == M_SWEEP) {
        if (epi && active) {
#pragma unroll 1
            for (int ch = 0; ch < CPT; ++ch) {
                const int o = 64 * (h * CPT + ch);
                float y[64];
                load_chunk(a.br + o, y);
                store_chunk(a.rstack + ((size_t)c * a.nr + (a.nr - 1)) * CHI + o, y);
            }
            if (h == 0) a.rexp[(size_t)c * a.nr + (a.nr - 1)] = 0;
        }
        start = (MODE == M_SWEEP && N == 1) ? a.bl : a.br;  // N = 1: no right-environment steps
        if (MODE == M_SWEEP) {
            pm = a.state[c].mant;
            pe = a.state[c].exp2;
        }
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tw = tmem + ((uint32_t)(q * 32) << 16);  // this warp's lanes
    const uint32_t ta = tw + (uint32_t)C::A_COL;             // their rows of A
    const uint32_t tm = tw + (uint32_t)C::META;              // their metadata
    Cursor cc = cursor_start<MODE>(a, j);
    // metadata of the next site (h = 0 warps): lane l carries the 16-bit slice
    // patterns of rows (l & 16) | (l & 7) and that row + 8 of its quadrant
    const int lane_a = (lane & 16) | (lane & 7), lane_b = lane_a | 8;
    auto write_meta = [&](const Cursor &x) {
        if (!epi || h != 0) return;
        const int sl = slice_of(x);
        const int s_a = __shfl_sync(FULL, sl, lane_a), s_b = __shfl_sync(FULL, sl, lane_b);
        tmem_st_1(tm, (s_a ? C::HALF1 : C::HALF0) | ((s_b ? C::HALF1 : C::HALF0) << 16));
        if (MODE == M_SWEEP && x.form == 0 && x.i == 0)  // the kept slice, second accumulator
            tmem_st_1(tm + (uint32_t)(C::META2 - C::META),
                      (s_a ? C::HALF0 : C::HALF1) | ((s_b ? C::HALF0 : C::HALF1) << 16));
    };
    // the exponent the renormalisation takes out of this row, held in the
    // accumulator at column col (first pass over the thread's chunks; kind:
    // exchange slot): max|v| brought into [1, 2), or 0 while every row of the
    // quadrant has its max in [1, 2^8) -- its 16-bit split stays inside FP16's
    // normal range with full precision relative to the max
    auto row_exp = [&](uint32_t col, int kind) -> int {
        float m8[8];
#pragma unroll 1
        for (int ch = 0; ch < CPT; ++ch) {
            float y[64];
            tmem_ld_64(tw + col + (uint32_t)(64 * (h * CPT + ch)), y);
#pragma unroll
            for (int i = 0; i < 64; ++i)
                m8[i & 7] = (ch == 0 && i < 8) ? fabsf(y[i]) : fmaxf(m8[i & 7], fabsf(y[i]));
        }
        const float part = fmaxf(fmaxf(fmaxf(m8[0], m8[1]), fmaxf(m8[2], m8[3])),
                                 fmaxf(fmaxf(m8[4], m8[5]), fmaxf(m8[6], m8[7])));
        const float mx = row_max(part, kind);
        const bool usable = (mx > 0.f) && isfinite(mx);
        int e = usable ? rttd::exponent_of(mx) : 0;
        if (__all_sync(FULL, !usable || (e >= 0 && e < 8)) || !usable) e = 0;
        return e;
    };
    // chunk ch of this thread (row entries o .. o + 63), scaled by 2^-e
    auto row_chunk = [&](uint32_t col, int e, int ch, float (&y)[64]) {
        tmem_ld_64(tw + col + (uint32_t)(64 * (h * CPT + ch)), y);
        scale_chunk(y, e);
    };
    // a row in global memory into the A operand
    auto write_A_row = [&](const float *src) {
#pragma unroll 1
        for (int ch = 0; ch < CPT; ++ch) {
            const int gc = h * CPT + ch;
            float y[64];
            load_chunk(src + 64 * gc, y);
            write_A_chunk<CHI, F16>(ta, gc, y);
        }
    };
    if (epi && total_steps > 0) {
        write_A_row(start);
        write_meta(cc);
    }
    tc_before();
    __syncthreads();
    tc_after();

    // producer (thread 0): cursor over atoms; atom g = step * KA + at
    long long g_issued = 0, g_waited = 0;
    Cursor pc = cursor_start<MODE>(a, j);
    int p_at = 0;
    auto issue_next = [&]() {
        const long long g = g_issued;
        const int st = (int)(g % NSG);
        const int y_hi = ((pc.form * 2 + 0) * a.L + pc.k) * CHI;
        const int y_lo = ((pc.form * 2 + 1) * a.L + pc.k) * CHI;
        const uint32_t dst = stage0 + (uint32_t)st * C::STAGE;
        mbar_expect_tx(full_bar(st), (uint32_t)C::STAGE);
        tma_load_2d(dst, &map, p_at * 64, y_hi, full_bar(st));
        tma_load_2d(dst + C::BOX, &map, p_at * 64, y_lo, full_bar(st));
        ++g_issued;
        if (++p_at == C::KA) {
            p_at = 0;
            cursor_next<MODE>(pc, a, span);
        }
    };
    if (issuer) {
        while (g_issued < total_atoms && g_issued < NSG) issue_next();
    }

    bool aborted = false;

    for (long long t = 0; t < total_steps; ++t) {
        const bool dbl = (MODE == M_SWEEP) && cc.form == 0 && cc.i == 0;
        // ---------------- MMA issue, then the refill (producer)
        if (issuer) {
            const uint32_t a_hi = tmem + (uint32_t)C::A_COL, a_lo = a_hi + (uint32_t)(CHI / 2);
            const uint32_t meta = tmem + (uint32_t)C::META;
            for (int at = 0; at < C::KA; ++at) {
                const long long g = t * C::KA + at;
                const int st = (int)(g % NSG);
                if (!mbar_wait(full_bar(st), (uint32_t)((g / NSG) & 1), a.wait_limit)) {
                    atomicOr(a.err, 1);
                    *abort_flag = 1;
                    break;
                }
                g_waited = g + 1;
                tc_after();
                const uint32_t b_hi = stage0 + (uint32_t)st * C::STAGE, b_lo = b_hi + C::BOX;
                // logical K [64 at + 32 kk, +32) reads row entries 32 at + 16 kk .. +16
                const uint64_t dh0 = sdesc(b_hi), dh1 = sdesc(b_hi + 64);
                const uint64_t dl0 = sdesc(b_lo), dl1 = sdesc(b_lo + 64);
                const uint32_t ao = (uint32_t)(at * 16);
                const uint32_t first = at != 0 ? 1u : 0u;
                mma_sp_ts(tmem, a_hi + ao, dh0, meta, C::IDESC, first);
                mma_sp_ts(tmem, a_hi + ao, dl0, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_lo + ao, dh0, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_hi + ao + 8, dh1, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_hi + ao + 8, dl1, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_lo + ao + 8, dh1, meta, C::IDESC, 1u);
                if (MODE == M_SWEEP && dbl) {  // the first site of a row: the kept slice too
                    const uint32_t d2 = tmem + (uint32_t)C::ACC2;
                    const uint32_t meta2 = tmem + (uint32_t)C::META2;
                    mma_sp_ts(d2, a_hi + ao, dh0, meta2, C::IDESC, first);
                    mma_sp_ts(d2, a_hi + ao, dl0, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_lo + ao, dh0, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_hi + ao + 8, dh1, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_hi + ao + 8, dl1, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_lo + ao + 8, dh1, meta2, C::IDESC, 1u);
                }
                mma_commit(empty_bar(st));
            }
            mma_commit(done_bar);
            // refill: each stage as soon as the MMAs that read it are done
            if (!*abort_flag) {
                for (int at = 0; at < C::KA; ++at) {
                    const long long g = t * C::KA + at;
                    if (g + NSG >= total_atoms) break;
                    const int st = (int)(g % NSG);
                    if (!mbar_wait(empty_bar(st), (uint32_t)((g / NSG) & 1), a.wait_limit)) {
                        atomicOr(a.err, 1);
                        *abort_flag = 1;
                        break;
                    }
                    issue_next();
                }
            }
        }
        bool write_next = false;
        const int k = cc.k;
        const int ck = site_cexp(k);
        const bool last = (t + 1 == total_steps);
        // ---------------- wait for the accumulator (epilogue warps)
        if (epi && !mbar_wait(done_bar, (uint32_t)(t & 1), a.wait_limit)) {
            atomicOr(a.err, 1);
            *abort_flag = 1;
        }
        tc_after();
        __syncwarp();
        // ---------------- epilogue
        if (!epi) {
            // the producer warp's other lanes only keep the cursor
        } else if (MODE != M_SWEEP || cc.form == 1) {
            // rows, amplitude, environments, and the sweep's right environment
            const int e = row_exp(0u, 0);
            E += e - ck;
            float *dst = nullptr;
            if (MODE == M_LEFT) {
                dst = a.lstack + ((size_t)c * N + k) * CHI;
                if (lead) a.lexp[(size_t)c * N + k] = (int32_t)E;
            } else if (MODE == M_RIGHT || MODE == M_SWEEP) {
                dst = a.rstack + ((size_t)c * a.nr + (k - rbase)) * CHI;
                if (lead) a.rexp[(size_t)c * a.nr + (k - rbase)] = (int32_t)E;
            }
            // the sweep's last right-environment step hands over to proposal 0 (from b_L)
            const bool to_bl = (MODE == M_SWEEP) && cc.tt == N - 2;
            write_next = (MODE == M_SWEEP) || !last;
            const bool closing = last && (MODE == M_ROWS || MODE == M_INIT);
            const float *rclose = a.br;
            if (closing) {
                fin_E = E;
                if (MODE == M_ROWS) {
                    const int rq = row_end(a, j) + 1 - a.kmin;  // r_{end+1}; b_R for j = N
                    rclose = a.rstack + ((size_t)c * a.nr + rq) * CHI;
                    fin_E = E + a.rexp[(size_t)c * a.nr + rq];
                }
            }
            float acc8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
            for (int ch = 0; ch < CPT; ++ch) {
                const int gc = h * CPT + ch;
                float y[64];
                row_chunk(0u, e, ch, y);
                if (dst && active) store_chunk(dst + 64 * gc, y);
                if (write_next && !to_bl) write_A_chunk<CHI, F16>(ta, gc, y);
                if (closing) dot_chunk(y, rclose + 64 * gc, acc8);
            }
            if (closing) fin_m = row_dot(dot_finish(acc8));
            if (to_bl) {
                write_A_row(a.bl);
                El = 0;
            }
        } else {  // M_SWEEP, a proposal row (form 0)
            const int jj = cc.jj;
            const int iq = site_spin(jj);
            const bool row_end_here = (cc.i + 1 == span);
            float acc8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const float *rr = a.rstack + ((size_t)c * a.nr + jj) * CHI;
            if (cc.i == 0) {
                // unflipped continuation: l_jj if the proposal is rejected
                const int e2 = row_exp((uint32_t)C::ACC2, 1);
                Ekeep = El + e2 - ck;
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    const int gc = h * CPT + ch;
                    float y[64];
                    row_chunk((uint32_t)C::ACC2, e2, ch, y);
                    if (active) store_chunk(a.lstack + ((size_t)c * N + jj) * CHI + 64 * gc, y);
                }
                if (lead) a.lexp[(size_t)c * N + jj] = (int32_t)Ekeep;
                // flipped start of the proposal row (kept for an acceptance)
                const int e1 = row_exp(0u, 0);
                Eflip = El + e1 - ck;
                E = Eflip;
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    const int gc = h * CPT + ch;
                    float y[64];
                    row_chunk(0u, e1, ch, y);
                    if (active) store_chunk(a.tmp + (size_t)c * CHI + 64 * gc, y);
                    if (!row_end_here) write_A_chunk<CHI, F16>(ta, gc, y);
                    else dot_chunk(y, rr + 64 * gc, acc8);
                }
                if (lead) a.tmp_exp[c] = (int32_t)Eflip;
            } else {
                const int e = row_exp(0u, 0);
                E += e - ck;
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    const int gc = h * CPT + ch;
                    float y[64];
                    row_chunk(0u, e, ch, y);
                    if (!row_end_here) write_A_chunk<CHI, F16>(ta, gc, y);
                    else dot_chunk(y, rr + 64 * gc, acc8);
                }
            }
            if (!row_end_here) {
                write_next = true;
            } else {
                // Metropolis decision of proposal jj (spin iq): every thread of
                // a row takes it from the same numbers
                double mm = row_dot(dot_finish(acc8));
                int64_t Ep = E + a.rexp[(size_t)c * a.nr + jj];
                normalize_scalar(mm, Ep);
                const double ratio = ldexp(mm / pm, (int)(Ep - pe));
                const double x = rttd::mcmc_uniform(a.seed, (uint64_t)(a.chain0 + c),
                                                    (uint64_t)(a.sweep0 + cc.sw), (uint64_t)jj);
                const bool accept = active && (x < ratio * ratio);
                if (accept) {
                    pm = mm;
                    pe = Ep;
                    ++acc_count;
                    El = Eflip;
                } else {
                    El = Ekeep;
                }
                if (h == 0) {
                    const uint32_t flips = __ballot_sync(FULL, accept);
                    if (lane == 0) bits[iq * 4 + q] ^= flips;
                    __syncwarp();
                }
                const bool next_prop = jj + 1 < N;
                const bool next_sweep = !next_prop && cc.sw + 1 < a.n_sweeps;
                // l_jj: the flipped start on acceptance (copied over the kept
                // row), else the kept row; the next proposal starts from it
                float *lj = a.lstack + ((size_t)c * N + jj) * CHI;
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    const int gc = h * CPT + ch;
                    float y[64];
                    load_chunk((accept ? a.tmp + (size_t)c * CHI : lj) + 64 * gc, y);
                    if (accept) store_chunk(lj + 64 * gc, y);
                    if (next_prop) write_A_chunk<CHI, F16>(ta, gc, y);
                }
                if (accept && h == 0) a.lexp[(size_t)c * N + jj] = (int32_t)Eflip;
                if (next_prop) {
                    write_next = true;
                } else if (next_sweep) {  // next sweep
                    write_A_row(N > 1 ? a.br : a.bl);
                    E = 0;
                    El = 0;
                    write_next = true;
                }
            }
        }
        cursor_next<MODE>(cc, a, span);
        if (write_next) write_meta(cc);
        tc_before();
        __syncthreads();
        tc_after();
        if (*abort_flag) {
            aborted = true;
            break;
        }
    }

    // a row with no site steps (the unflipped row when every site lies in the
    // first block, R = 1) closes on its start row
    if (MODE == M_ROWS && total_steps == 0 && epi) {
        const int rq = row_end(a, j) + 1 - a.kmin;
        const float *rclose = a.rstack + ((size_t)c * a.nr + rq) * CHI;
        fin_E = E + a.rexp[(size_t)c * a.nr + rq];
        float acc8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int ch = 0; ch < CPT; ++ch) {
            const int gc = h * CPT + ch;
            float y[64];
            load_chunk(start + 64 * gc, y);
            dot_chunk(y, rclose + 64 * gc, acc8);
        }
        fin_m = row_dot(dot_finish(acc8));
    }
    // ---------------- outputs
    if (!aborted && lead) {
        if (MODE == M_ROWS) {
            double mm = fin_m;
            int64_t Ep = fin_E;
            normalize_scalar(mm, Ep);
            a.rows_mant[c * (N + 1) + j] = mm;
            a.rows_exp[c * (N + 1) + j] = Ep;
        } else if (MODE == M_INIT) {
            double mm = fin_m;
            int64_t Ep = fin_E;
            normalize_scalar(mm, Ep);
            if (a.state) {
                a.state[c].mant = mm;
                a.state[c].exp2 = Ep;
            }
            if (a.log_abs)
                a.log_abs[c] = (mm == 0.0) ? -INFINITY : (double)Ep * 0.6931471805599453 + log(fabs(mm));
            if (a.sign) a.sign[c] = (mm > 0.0) ? 1 : ((mm < 0.0) ? -1 : 0);
        } else if (MODE == M_SWEEP) {
            for (int i = 0; i < N; ++i) a.spins_out[c * N + i] = (uint8_t)spin(i);
            a.state[c].mant = pm;
            a.state[c].exp2 = pe;
            if (a.n_accept) a.n_accept[c] += acc_count;
        }
    }
    // ---------------- teardown: drain own copies (bounded), free TMEM
    if (issuer && aborted) {
        for (long long g = g_waited; g < g_issued; ++g)
            mbar_wait(full_bar((int)(g % NSG)), (uint32_t)((g / NSG) & 1), a.wait_limit);
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tmem_dealloc(tmem, TALLOC);
}

// ------------------------------------------------------------------ failure-detection self-test
// A bounded wait that nothing completes: one warp allocates tensor memory,
// arms an mbarrier that no copy and no MMA will ever arrive on, waits on it
// with the given clock budget, records bit 0 in the error word when the
// budget runs out (as every wait of the sampler's kernels does), frees its
// tensor memory and returns.  Nothing asynchronous is in flight at any time.
__global__ void __launch_bounds__(32, 1) k_wait_selftest(int *err, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    tmem_alloc(sa(&slot), 32);
    if (threadIdx.x == 0) {
        mbar_init(sa(&bar), 1);
        fence_barrier_init();
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = slot;
    if (threadIdx.x == 0 && !mbar_wait(sa(&bar), 0u, limit)) atomicOr(err, 1);
    tc_before();
    __syncthreads();
    tc_after();
    tmem_dealloc(tmem, 32);
}

// ------------------------------------------------------------------ split-row sweep (chi = 64)
// Each proposal row psi(s') = l_{j-1} A_j' ... A_m . (A_{m+1} ... A'_{(R-1)N+j} r)
// is computed as two half-rows at once: the left tile walks sites j..m from
// l_{j-1} (left to right), the right tile walks (R-1)N+j..m+1 from the cached
// right environment (right to left); the halves meet in one dot product and
// the Metropolis decision.  The two tiles run on the two CTAs of a cluster
// (k_tc_sweep_pair below).  On a general path (GEN) proposal j's row covers
// sites j..L-1 (spin p[j] flipped wherever it sits); the left tile walks the
// first half from l_{j-1}, the right tile the second half backwards from b_R
// with the current spins, so no right environment is kept.
constexpr int SP_HAND = 64 * NT * 4;  // right half-rows, [64][128] floats

__device__ __forceinline__ void named_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// GEN: a general path.  Proposal j's row covers sites j..L-1 (spin p[j]
// flipped wherever it sits); the left tile walks the first half from l_{j-1},
// the right tile the second half backwards from b_R with the current spins,
// so no right environment is kept.


// ------------------------------------------------------------------ two epilogue warps per row group
// The epilogue of a tile is spread over 8 warps: warp (quadrant q, half h)
// owns rows 32q..32q+31 (TMEM lanes of quadrant q) and the columns
// [32h, 32h+32) of every row.  The two warps of a quadrant meet in a
// 64-thread named barrier to combine the row maximum of each site and the
// partial dot product of each decision, through shared-memory slots
// double-buffered by the exchange count.  Both halves of a row take the same
// scale: the lazy-rescale vote of a warp covers the same 32 rows in both
// warps.

// Store 16 columns at t0 and 16 at t1 of this warp's 32 TMEM lanes, then wait.
__device__ __forceinline__ void tmem_st_2x16(uint32_t t0, uint32_t t1, const uint32_t (&x)[16],
                                             const uint32_t (&y)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%1], {%18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(t0), "r"(t1), "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]), "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), "r"(x[14]), "r"(x[15]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(y[7]), "r"(y[8]), "r"(y[9]), "r"(y[10]), "r"(y[11]), "r"(y[12]), "r"(y[13]), "r"(y[14]), "r"(y[15])
        : "memory");
}

// Columns [32h, 32h+32) of the accumulator slice `sel` of this warp's lanes.
__device__ __forceinline__ void acc_select_half(uint32_t tw, int h, int sel, float (&v)[32]) {
    uint32_t x0[32], x1[32];
    tmem_ld_2x32(tw + (uint32_t)(32 * h), tw + 64u + (uint32_t)(32 * h), x0, x1);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(sel ? x1[i] : x0[i]);
}

__device__ __forceinline__ float half_max(const float (&v)[32]) {
    float m[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) m[p] = fabsf(v[p]);
#pragma unroll
    for (int i = 8; i < 32; ++i) m[i & 7] = fmaxf(m[i & 7], fabsf(v[i]));
    return fmaxf(fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3])),
                 fmaxf(fmaxf(m[4], m[5]), fmaxf(m[6], m[7])));
}

// renorm of a half row given the whole row's maximum (see renorm).
__device__ __forceinline__ int renorm_half(float (&v)[32], float mx) {
    const bool usable = (mx > 0.f) && isfinite(mx);
    const int e = usable ? rttd::exponent_of(mx) : 0;
    if (__all_sync(FULL, !usable || (e >= 0 && e < 8))) return 0;
    if (!usable) return 0;
    if (rttd::pow2_normal(0.f, -e)) {
        const float sc = rttd::pow2(0.f, -e);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] *= sc;
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = rttd::scale2(v[i], -e);
    }
    return e;
}

// Half h of row m as the A operand: entries 32h..32h+31 in columns 16h.. of
// the hi block at ta and of the lo block at ta + 32.
template <bool F16>
__device__ __forceinline__ void write_A_half(uint32_t ta, int h, const float (&v)[32]) {
    uint32_t hh[16], ll[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) split2<F16>(v[2 * p], v[2 * p + 1], hh[p], ll[p]);
    tmem_st_2x16(ta + (uint32_t)(16 * h), ta + 32u + (uint32_t)(16 * h), hh, ll);
}



// ------------------------------------------------------------------ split-row sweep on a CTA pair
// The two half-row tiles on the two CTAs of a cluster (rank 0 left, rank 1
// right), i.e. on two SMs with a tensor pipe each, each tile's epilogue on two
// warps per row group (above).  Per
// proposal the right CTA stores its finished half-row (and exponent) into the
// left CTA's shared memory and arrives on the left's `hand` mbarrier; the left
// decides, stores the flip bits into the right CTA's spin bits and arrives on
// the right's `decision` mbarrier (release/acquire at cluster scope).  Every
// wait is bounded; both CTAs meet in a cluster barrier before they exit.
// Roles per CTA: warps 0-7 epilogue (two per TMEM lane quadrant), warp 8 MMA
// issuer, warp 9 TMA loads.  TMEM (left): accumulator [0,128), first-site
// accumulator [128,256), A hi/lo [256,320); (right): accumulator [0,128), A
// hi/lo [128,192).
constexpr int SPC_THREADS = 320;

// Float-float arithmetic for the pair sweep's Metropolis decision (GB300's FP64
// rate is 1/64 of FP32; a warp-wide FP64 instruction costs ~64 issue cycles on
// the decision's critical path).  two_sum is Knuth's error-free addition.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (h, l) <- (h, l) + (h2, l2), renormalised so that |l| <= ulp(h)/2
__device__ __forceinline__ void ff_add(float &h, float &l, float h2, float l2) {
    float s, e;
    two_sum(h, h2, s, e);
    e += l + l2;
    h = s + e;
    l = e - (h - s);
}
// The Metropolis uniform of (chain, sweep, proposal) cut to its top 24 bits, as
// a float in [0, 1): the 53-bit uniform minus less than 2^-24.
__device__ __forceinline__ float mcmc_uniform24(uint64_t seed, uint64_t chain, uint64_t sweep,
                                                uint64_t proposal) {
    uint64_t x[4];
    rttd::philox4x64_10(chain, sweep, proposal, 0ull, seed, 0x4D434D43ull, x);
    return (float)(uint32_t)(x[0] >> 40) * 0x1.0p-24f;
}
// sites the left tile takes below half of a proposal's row; negative: more.
// Measured on plain_6x6 (37 sites per row): -1 (19 left, 18 right) is fastest;
// the right tile also hands its half-row over and waits for the decision.
constexpr int kPairLeftLess = -1;

inline size_t sweepc_smem(int N, int L) {
    return 1024 + (size_t)NS * Cfg<64>::STAGE + SP_HAND + 256 + (size_t)16 * N + (size_t)4 * L +
           16 + 4 * NT + 16 + (size_t)2 * 2 * NT * 4 + (size_t)2 * 2 * NT * 8;
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
    return out;
}
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, long long limit) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_cluster(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// Bulk copy (copy engine) of `bytes` from this CTA's shared memory to a peer
// CTA's, completing as transaction bytes on the peer's mbarrier.
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t dst_cluster, uint32_t src_cta,
                                                  uint32_t bytes, uint32_t mbar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_cluster),
        "r"(src_cta), "r"(bytes), "r"(mbar_cluster)
        : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

template <bool F16, bool GEN>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(SPC_THREADS, 1)
    k_tc_sweep_pair(const __grid_constant__ CUtensorMap map, const Args a) {
    constexpr int CHI = 64;
    using C = Cfg<CHI, F16>;
    extern __shared__ uint8_t smem_raw[];
    // the dynamic shared memory starts at the same offset in both CTAs, so the
    // 1024-byte alignment below gives the same layout in both
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t ring0 = sa(base);
    float *hand = (float *)(base + NS * C::STAGE);  // [128 rows][64], float4 chunks swizzled
    uint64_t *bars = (uint64_t *)(base + NS * C::STAGE + SP_HAND);
    const uint32_t bar0 = sa(bars);
    // bars: full[NS], empty[NS], done, hand (left), decision (right)
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (NS + s); };
    const uint32_t done_bar = bar0 + 8u * (2 * NS);
    const uint32_t hand_bar = bar0 + 8u * (2 * NS + 1);
    const uint32_t dec_bar = bar0 + 8u * (2 * NS + 2);
    uint32_t *tmem_slot = (uint32_t *)(bars + 8);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    long long *issued = (long long *)(bars + 10);
    uint32_t *bits = (uint32_t *)(base + NS * C::STAGE + SP_HAND + 256);
    uint32_t *tab = bits + 4 * a.N;
    int32_t *rexp_s = (int32_t *)(((uintptr_t)(tab + a.L) + 15) & ~(uintptr_t)15);  // 16-aligned
    // exchange slots, 16-byte aligned whatever L is
    float *xmax = (float *)(((uintptr_t)(rexp_s + NT) + 15) & ~(uintptr_t)15);  // [parity][half][row]
    double *xdot = (double *)(xmax + 2 * 2 * NT);                              // [parity][half][row]

    // one hand-off: the right half-rows (128 x 64 floats) and their exponents
    constexpr uint32_t HAND_BYTES = (uint32_t)SP_HAND + 4u * NT;
    const uint32_t rank = cluster_rank();
    const int X = (int)rank;  // 0 left, 1 right
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.N, L = a.L;
    const int span = (a.R - 1) * N + 1;
    auto nL_of = [&](int j) -> int {
        const int T = GEN ? L - j : span;
        return min(T - 1, max(1, T / 2 - kPairLeftLess));
    };
    auto nR_of = [&](int j) -> int { return (GEN ? L - j : span) - nL_of(j); };
    const int q = warp & 3, hf = (warp >> 2) & 1;
    const int m = q * 32 + lane;
    const int64_t c_raw = (int64_t)(blockIdx.x >> 1) * NT + m;
    const bool active = c_raw < a.B;
    const int64_t c = active ? c_raw : a.B - 1;
    const uint32_t tcols = X == 0 ? 512u : 256u;

    if (warp == 0) tmem_alloc(sa(tmem_slot), tcols);
    if (tid == 0) {
        for (int i = 0; i < 2 * NS + 1; ++i) mbar_init(bar0 + 8u * i, 1);
        mbar_init(hand_bar, 1);  // armed by the left with the bytes of one hand-off
        mbar_init(dec_bar, 8);   // one arrival per left epilogue warp
        *abort_flag = 0;
        issued[0] = 0;
        fence_barrier_init();
        if (X == 0) mbar_expect_tx(hand_bar, HAND_BYTES);  // the first proposal's hand-off
    }
    for (int k = tid; k < L; k += SPC_THREADS)
        tab[k] = ((uint32_t)__ldg(GEN ? a.path + k : a.q + (k % N)) & 0xffffu) |
                 ((uint32_t)(__ldg(a.cexp + k) & 0xffff) << 16);
    if (warp < 4) {
        for (int i = 0; i < N; ++i) {
            const uint32_t w = __ballot_sync(FULL, a.spins_in[c * N + i] != 0);
            if (lane == 0) bits[i * 4 + warp] = w;
        }
    }
    tc_before();
    cluster_sync_all();  // barriers initialised in both CTAs before any remote arrive
    tc_after();
    const uint32_t tmem = *tmem_slot;
    auto spin = [&](int i) -> int { return (int)((bits[i * 4 + q] >> lane) & 1u); };
    auto site_spin = [&](int k) -> int { return (int)(tab[k] & 0xffffu); };
    auto site_cexp = [&](int k) -> int { return (int)(int16_t)(tab[k] >> 16); };
    auto fail_now = [&]() {
        atomicOr(a.err, 1);
        *abort_flag = 1;
    };
    auto bwait = [&](uint32_t bar, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (!mbar_wait(bar, parity, a.wait_limit)) {
            fail_now();
            return false;
        }
        return true;
    };
    auto bwait_cluster = [&](uint32_t bar, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (!mbar_wait_cluster(bar, parity, a.wait_limit)) {
            fail_now();
            return false;
        }
        return true;
    };
    auto publish = [&]() {
        tc_before();
        named_arrive(2, 2 * NT + 32);
    };
    int xpar = 0;
    auto pair_max = [&](float mine) -> float {
        float *slot = xmax + (xpar * 2) * NT;
        slot[hf * NT + m] = mine;
        named_sync(4 + q, 64);
        const float other = slot[(hf ^ 1) * NT + m];
        xpar ^= 1;
        return fmaxf(mine, other);
    };
    // the two halves' partial dot products as float-float pairs, summed in
    // the same order by both warps
    int dpar = 0;
    auto pair_dot = [&](float mh, float ml, float &h, float &l) {
        float2 *slot = reinterpret_cast<float2 *>(xdot) + (dpar * 2) * NT;
        slot[hf * NT + m] = make_float2(mh, ml);
        named_sync(4 + q, 64);
        const float2 d0 = slot[m], d1 = slot[NT + m];
        dpar ^= 1;
        h = d0.x;
        l = d0.y;
        ff_add(h, l, d1.x, d1.y);
    };
    const uint32_t acc_col = 0u, t0_col = 128u, a_col = X == 0 ? 256u : 128u;

    if (warp == 8) {
        // ---------------------------------------------------------- MMA issuer
        long long g = 0;
        auto issue = [&](uint32_t dcol) {
            named_sync(2, 2 * NT + 32);
            if (lane == 0) {
                const int s = (int)(g % NS);
                if (bwait(full_bar(s), (uint32_t)((g / NS) & 1))) {
                    tc_after();
                    const uint32_t ahi = tmem + a_col, alo = ahi + 32u;
                    const uint32_t b_hi = ring0 + (uint32_t)s * C::STAGE, b_lo = b_hi + C::BOX;
                    const uint32_t d = tmem + dcol;
#pragma unroll
                    for (int kb = 0; kb < 4; ++kb) {
                        const uint32_t o = (uint32_t)(kb * 32), ka = (uint32_t)(kb * 8);
                        mma_f16_ts(d, ahi + ka, sdesc(b_hi + o), C::IDESC, kb != 0 ? 1u : 0u);
                        mma_f16_ts(d, ahi + ka, sdesc(b_lo + o), C::IDESC, 1u);
                        mma_f16_ts(d, alo + ka, sdesc(b_hi + o), C::IDESC, 1u);
                    }
                    mma_commit(empty_bar(s));
                    mma_commit(done_bar);
                }
            }
            ++g;
            __syncwarp();
        };
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            if (X == 1) {
                if (!GEN)
                    for (int u = 0; u < N - 1; ++u) issue(acc_col);
                for (int j = 0; j < N; ++j)
                    for (int t = 0; t < nR_of(j); ++t) issue(acc_col);
            } else {
                for (int j = 0; j < N; ++j)
                    for (int t = 0; t < nL_of(j); ++t) issue(t == 0 ? t0_col : acc_col);
            }
        }
    } else if (warp == 9) {
        // ---------------------------------------------------------- TMA loads
        if (lane == 0) {
            long long n = 0;
            auto load = [&](int k) {
                const long long g = n++;
                const int s = (int)(g % NS);
                if (*abort_flag) return;
                if (g >= NS && !bwait(empty_bar(s), (uint32_t)(((g / NS) - 1) & 1))) return;
                const int y_hi = ((X * 2 + 0) * L + k) * 2 * CHI;
                const int y_lo = ((X * 2 + 1) * L + k) * 2 * CHI;
                const uint32_t dst = ring0 + (uint32_t)s * C::STAGE;
                mbar_expect_tx(full_bar(s), (uint32_t)C::STAGE);
                tma_load_2d(dst, &map, 0, y_hi, full_bar(s));
                tma_load_2d(dst + C::BOX, &map, 0, y_lo, full_bar(s));
                issued[0] = g + 1;
            };
            for (int sw = 0; sw < a.n_sweeps; ++sw) {
                if (X == 1 && !GEN)
                    for (int u = 0; u < N - 1; ++u) load(L - 1 - u);
                for (int j = 0; j < N; ++j) {
                    if (X == 0)
                        for (int t = 0; t < nL_of(j); ++t) load(j + t);
                    else
                        for (int t = 0; t < nR_of(j); ++t) load(GEN ? L - 1 - t : (a.R - 1) * N + j - t);
                }
            }
        }
    } else if (X == 0) {
        // ---------------------------------------------------------- left epilogue
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        const uint32_t tw = tq + acc_col, tw0 = tq + t0_col, ta = tq + a_col;
        const uint32_t peer_dec = peer_addr(dec_bar, 1u);
        float v[32];
        load_vec<32>(a.bl + 32 * hf, v);
        write_A_half<F16>(ta, hf, v);
        publish();
        // the chain amplitude as a float-float mantissa (|pm_h| in [1,2)) and
        // an exact exponent; converted back to FP64 once, at the end
        const double pm0 = a.state[c].mant;
        float pm_h = (float)pm0, pm_l = (float)(pm0 - (double)pm_h);
        int64_t pe = a.state[c].exp2, acc_count = 0;
        int64_t El = 0, E = 0;
        long long nd = 0, np = 0;
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            for (int j = 0; j < N; ++j) {
                const int iq = site_spin(j);
                const int si = spin(iq);
                const int nL = nL_of(j);
                float x = 0.f;
                float mx_keep = 0.f, mx_flip = 0.f;
                for (int t = 0; t < nL; ++t) {
                    const int k = j + t;
                    bwait(done_bar, (uint32_t)(nd++ & 1));
                    tc_after();
                    __syncwarp();
                    const int sk = site_spin(k);
                    if (t == 0) {
                        float vk[32];
                        acc_select_half(tw0, hf, si, vk);
                        acc_select_half(tw0, hf, si ^ 1, v);
                        const float a0 = half_max(vk), a1 = half_max(v);
                        mx_keep = pair_max(a0);
                        mx_flip = pair_max(a1);
                        E = El + renorm_half(v, mx_flip) - site_cexp(k);
                    } else {
                        acc_select_half(tw, hf, spin(sk) ^ (sk == iq ? 1 : 0), v);
                        E += renorm_half(v, pair_max(half_max(v))) - site_cexp(k);
                    }
                    if (t + 1 < nL) {
                        write_A_half<F16>(ta, hf, v);
                        publish();
                    }
                    if (t == 0)
                        x = mcmc_uniform24(a.seed, (uint64_t)(a.chain0 + c),
                                           (uint64_t)(a.sweep0 + sw), (uint64_t)j);
                }
                // the right half-row, from the peer CTA; then arm the next hand-off
                bwait_cluster(hand_bar, (uint32_t)(np++ & 1));
                if (tid == 0 && (j + 1 < N || sw + 1 < a.n_sweeps)) mbar_expect_tx(hand_bar, HAND_BYTES);
                // psi(s') = (mm_h + mm_l) 2^Ep: eight FP32 partial dot products per
                // half, added without error (float-float)
                float mm_h, mm_l;
                {
                    float acc[8];
#pragma unroll
                    for (int p = 0; p < 8; ++p) acc[p] = 0.f;
#pragma unroll
                    for (int cc = 0; cc < 8; ++cc) {
                        const int ch = hf * 8 + cc;  // float4 chunk of row m
                        const float4 w = *reinterpret_cast<const float4 *>(
                            hand + m * 64 + ((ch ^ (m & 15)) << 2));
                        acc[(4 * cc) & 7] = fmaf(v[4 * cc], w.x, acc[(4 * cc) & 7]);
                        acc[(4 * cc + 1) & 7] = fmaf(v[4 * cc + 1], w.y, acc[(4 * cc + 1) & 7]);
                        acc[(4 * cc + 2) & 7] = fmaf(v[4 * cc + 2], w.z, acc[(4 * cc + 2) & 7]);
                        acc[(4 * cc + 3) & 7] = fmaf(v[4 * cc + 3], w.w, acc[(4 * cc + 3) & 7]);
                    }
                    float ph = acc[0], pl = 0.f;
#pragma unroll
                    for (int p = 1; p < 8; ++p) ff_add(ph, pl, acc[p], 0.f);
                    pair_dot(ph, pl, mm_h, mm_l);
                }
                int64_t Ep = E + rexp_s[m];
                if (mm_h != 0.f && isfinite(mm_h)) {  // |mm_h| into [1,2), exactly
                    const int kk = rttd::exponent_of(mm_h);
                    mm_h = rttd::scale2(mm_h, -kk);
                    mm_l = rttd::scale2(mm_l, -kk);
                    Ep += kk;
                }
                // accept iff u < (psi'/psi)^2, i.e. u < q^2 4^d with q = mm/pm in
                // (1/2, 2) and d = Ep - pe; FP32 (the split path's ratios carry
                // errors far above the rounding of q^2)
                bool pass;
                {
                    const float qq = mm_h / pm_h;
                    const int64_t d = Ep - pe;
                    if (!(mm_h != 0.f && isfinite(mm_h)))
                        pass = false;  // a zero or undefined proposal is never taken
                    else if (pm_h == 0.f || !isfinite(pm_h))
                        pass = true;   // a chain at psi = 0 takes any finite nonzero one
                    else if (d >= 1)
                        pass = true;
                    else if (d < -75)
                        pass = false;
                    else
                        pass = x < ldexpf(qq * qq, (int)(2 * d));
                }
                const bool accept = active && !*abort_flag && pass;
                if (accept) {
                    pm_h = mm_h;
                    pm_l = mm_l;
                    pe = Ep;
                    ++acc_count;
                }
                const uint32_t flips = __ballot_sync(FULL, accept);
                if (lane == 0 && hf == 0) {
                    const uint32_t w = bits[iq * 4 + q] ^ flips;
                    bits[iq * 4 + q] = w;
                    st_cluster_u32(peer_addr(sa(bits + iq * 4 + q), 1u), w);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(peer_dec);  // the decision is with the right CTA
                acc_select_half(tw0, hf, si ^ (accept ? 1 : 0), v);
                El += renorm_half(v, accept ? mx_flip : mx_keep) - site_cexp(j);
                const bool more = (j + 1 < N) || (sw + 1 < a.n_sweeps);
                if (j + 1 < N) {
                    write_A_half<F16>(ta, hf, v);
                    publish();
                }
                if (j + 1 == N && more) {
                    load_vec<32>(a.bl + 32 * hf, v);
                    El = 0;
                    write_A_half<F16>(ta, hf, v);
                    publish();
                }
            }
        }
        // after an expired wait: let a hand-off that is still in flight land
        if (tid == 0 && *abort_flag) mbar_wait_cluster(hand_bar, (uint32_t)(np & 1), a.wait_limit);
        if (active && !*abort_flag && hf == 0) {
            double pm = (double)pm_h + (double)pm_l;
            normalize_scalar(pm, pe);
            a.state[c].mant = pm;
            a.state[c].exp2 = pe;
            if (a.n_accept) a.n_accept[c] += acc_count;
        }
    } else {
        // ---------------------------------------------------------- right epilogue
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        const uint32_t tw = tq + acc_col, ta = tq + a_col;
        const uint32_t peer_hand = peer_addr(hand_bar, 0u);
        const uint32_t peer_rows = peer_addr(sa(hand), 0u);
        const uint32_t peer_rexp = peer_addr(sa(rexp_s), 0u);
        float v[32];
        load_vec<32>(a.br + 32 * hf, v);
        if (active && !GEN) {
            store_vec<32>(a.rstack + ((size_t)c * N + (N - 1)) * CHI + 32 * hf, v);
            if (hf == 0) a.rexp[(size_t)c * N + (N - 1)] = 0;
        }
        write_A_half<F16>(ta, hf, v);
        publish();
        int64_t E = 0;
        long long nd = 0, ndec = 0;
        // The left's decision on proposal j changes only spin p(j): wait for it
        // (its spin bits arrive with it) before the first select at a site that
        // carries that spin, and before this CTA's hand-off buffer is rewritten
        // (the left has consumed the previous hand-off once it decides).
        int pend = -1;
        auto settle = [&]() {
            if (pend >= 0) {
                bwait_cluster(dec_bar, (uint32_t)(ndec++ & 1));
                pend = -1;
            }
        };
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            E = 0;
            for (int u = 0; u < (GEN ? 0 : N - 1); ++u) {
                const int k = L - 1 - u;
                bwait(done_bar, (uint32_t)(nd++ & 1));
                tc_after();
                __syncwarp();
                if (site_spin(k) == pend) settle();
                acc_select_half(tw, hf, spin(site_spin(k)), v);
                E += renorm_half(v, pair_max(half_max(v))) - site_cexp(k);
                if (active) {
                    store_vec<32>(a.rstack + ((size_t)c * N + (k - (a.R - 1) * N - 1)) * CHI + 32 * hf, v);
                    if (hf == 0) a.rexp[(size_t)c * N + (k - (a.R - 1) * N - 1)] = (int32_t)E;
                }
                write_A_half<F16>(ta, hf, v);
                publish();
            }
            for (int j = 0; j < N; ++j) {
                const int iq = site_spin(j);
                const int nR = nR_of(j);
                if (GEN)
                    E = 0;
                else if (j > 0)
                    E = a.rexp[(size_t)c * N + j];
                for (int t = 0; t < nR; ++t) {
                    const int k = GEN ? L - 1 - t : (a.R - 1) * N + j - t;
                    bwait(done_bar, (uint32_t)(nd++ & 1));
                    tc_after();
                    __syncwarp();
                    const int sk = site_spin(k);
                    if (sk == pend) settle();
                    acc_select_half(tw, hf, spin(sk) ^ (sk == iq ? 1 : 0), v);
                    E += renorm_half(v, pair_max(half_max(v))) - site_cexp(k);
                    if (t + 1 < nR) {
                        write_A_half<F16>(ta, hf, v);
                        publish();
                    }
                }
                settle();  // the previous hand-off has been read
                // hand the half-row to the left CTA: row m (float4 chunks 8hf..8hf+7)
                // into this CTA's buffer, then one bulk copy of all rows and exponents
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    const int ch = hf * 8 + cc;
                    *reinterpret_cast<float4 *>(hand + m * 64 + ((ch ^ (m & 15)) << 2)) =
                        make_float4(v[4 * cc], v[4 * cc + 1], v[4 * cc + 2], v[4 * cc + 3]);
                }
                if (hf == 0) rexp_s[m] = (int32_t)E;
                fence_async_smem();
                named_sync(1, 2 * NT);  // the 8 epilogue warps have written
                if (tid == 0 && !*abort_flag) {
                    bulk_copy_to_peer(peer_rows, sa(hand), (uint32_t)SP_HAND, peer_hand);
                    bulk_copy_to_peer(peer_rexp, sa(rexp_s), 4u * NT, peer_hand);
                }
                const bool more = (j + 1 < N) || (sw + 1 < a.n_sweeps);
                if (more) {  // the next row's first MMA does not depend on this decision
                    if (j + 1 < N && !GEN)
                        load_vec<32>(a.rstack + ((size_t)c * N + (j + 1)) * CHI + 32 * hf, v);
                    else
                        load_vec<32>(a.br + 32 * hf, v);
                    write_A_half<F16>(ta, hf, v);
                    publish();
                }
                pend = iq;  // this proposal's decision is now outstanding
            }
        }
        settle();
    }
    __syncthreads();
    if (X == 0 && warp < 4 && active && !*abort_flag) {
        for (int i = 0; i < N; ++i) a.spins_out[c * N + i] = (uint8_t)spin(i);
    }
    if (tid == 0 && *abort_flag) {
        for (long long g = (issued[0] > NS ? issued[0] - NS : 0); g < issued[0]; ++g)
            mbar_wait(full_bar((int)(g % NS)), (uint32_t)((g / NS) & 1), a.wait_limit);
    }
    tc_before();
    cluster_sync_all();  // no CTA leaves while its peer may still store into it
    tc_after();
    if (warp == 0) tmem_dealloc(tmem, tcols);
}


// ------------------------------------------------------------------ split-row sweep (chi = 128)
// The chi = 128 sweep on a CTA pair, with the sparse site products of k_tc:
// each proposal row is split between a left tile (sites j..j+nL-1 from
// l_{j-1}, rank 0) and a right tile (the rest, backwards from the cached
// right environment, rank 1), each on its own SM with its own tensor pipe and
// tensor memory, so a proposal costs about half the sequential site steps of
// the single-tile sweep and a batch holds twice the SMs.  Per CTA: four
// epilogue warps (one row per thread, 64-column chunks) and one producer warp
// whose lane 0 streams the site tensors by TMA and issues the MMAs.
//   left : first site of a row into two accumulators (flipped slice, the kept
//          slice = l_j if rejected); at its last site it waits for the right
//          half-row, forms psi(s') by one dot product, decides (R8: FP64
//          ratio, 53-bit uniform), keeps the flip bits and stores them into
//          the right CTA's spin words, then arrives on the right's decision
//          barrier (release / acquire at cluster scope).
//   right: per sweep the right environment r_k (last block), then per
//          proposal its half-row; the finished half-row (FP32, 128 x 128,
//          float4 chunks swizzled by row) and its exponents go to the left
//          CTA's shared memory in one bulk copy completing on the left's
//          mbarrier.  It waits for the left's decision on spin p(j) only
//          before the metadata of a site that carries that spin, and before
//          it rewrites its hand-off buffer.
// TMEM (512 columns in both): accumulator [0,128), kept accumulator
// [128,256) (left), A hi/lo [256,384), metadata at 384 and 448.  Every wait is
// bounded; both CTAs meet in a cluster barrier before they exit.
constexpr int SPP_THREADS = NT + 32;
constexpr int SPP_HAND = NT * 128 * 4;        // one right half-row hand-off, [128][128] floats
constexpr int kPairLeftLess128 = 1;           // sites the left tile takes below half a row

inline size_t spp_smem(int N, int L) {
    return 1024 + (size_t)SCfg<128>::NSTG * SCfg<128>::STAGE + SPP_HAND + 4 * NT + 128 +
           (size_t)16 * N + (size_t)4 * L;
}

// Chunk ch (entries 64 ch .. 64 ch + 63) of the closing contraction against
// the hand-off buffer (row m, float4 chunk x at ((x ^ (m & 7)) << 2)), in the
// partial sums dot_chunk uses.
__device__ __forceinline__ void dot_hand(const float (&y)[64], const float *__restrict__ hrow, int m,
                                         int ch, float (&acc)[8]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float4 x = *reinterpret_cast<const float4 *>(hrow + (((16 * ch + i) ^ (m & 7)) << 2));
        const int p = (2 * i) & 7;
        acc[p] = fmaf(y[4 * i], x.x, acc[p]);
        acc[p + 1] = fmaf(y[4 * i + 1], x.y, acc[p + 1]);
        acc[(p + 2) & 7] = fmaf(y[4 * i + 2], x.z, acc[(p + 2) & 7]);
        acc[(p + 3) & 7] = fmaf(y[4 * i + 3], x.w, acc[(p + 3) & 7]);
    }
}
__device__ __forceinline__ void put_hand(const float (&y)[64], float *__restrict__ hrow, int m, int ch) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
        *reinterpret_cast<float4 *>(hrow + (((16 * ch + i) ^ (m & 7)) << 2)) =
            make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
}

// Position of a CTA in its sequence of site steps: sweep, proposal, step of
// the half-row (or of the right environment when env is set).
struct PairCur {
    int sw, j, t, env;
};

template <bool F16, bool GEN>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(SPP_THREADS, 1)
    k_sp_pair(const __grid_constant__ CUtensorMap map, const Args a) {
    constexpr int CHI = 128;
    using C = SCfg<CHI, F16>;
    static_assert(C::NH == 1 && C::CPT == 2, "one epilogue thread per row");
    constexpr int NSG = C::NSTG;
    constexpr int CPT = C::CPT;
    constexpr uint32_t HAND_BYTES = (uint32_t)SPP_HAND + 4u * NT;
    extern __shared__ uint8_t smem_raw[];
    // the dynamic shared memory starts at the same offset in both CTAs, so the
    // 1024-byte alignment gives the same layout in both
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t stage0 = sa(base);
    float *hand = (float *)(base + NSG * C::STAGE);      // [128][128] (+ exponents below)
    int32_t *hexp = (int32_t *)(hand + NT * CHI);        // [128]
    uint64_t *bars = (uint64_t *)(hexp + NT);
    const uint32_t bar0 = sa(bars);
    // bars: full[NSG], empty[NSG], done, hand (left), decision (right)
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (NSG + s); };
    const uint32_t done_bar = bar0 + 8u * (2 * NSG);
    const uint32_t hand_bar = bar0 + 8u * (2 * NSG + 1);
    const uint32_t dec_bar = bar0 + 8u * (2 * NSG + 2);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NSG + 3);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    uint32_t *bits = (uint32_t *)((uint8_t *)bars + 128);
    uint32_t *tab = bits + 4 * a.N;

    const int X = (int)cluster_rank();  // 0 left, 1 right
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool epi = warp < 4;
    const bool issuer = warp == 4 && lane == 0;
    const int q = warp & 3;
    const int m = 32 * q + lane;
    const int64_t c_raw = (int64_t)(blockIdx.x >> 1) * NT + m;
    const bool active = epi && c_raw < a.B;
    const int64_t c = c_raw < a.B ? c_raw : a.B - 1;
    const int N = a.N, L = a.L;
    const int span = (a.R - 1) * N + 1;
    const int rbase = a.kmin;
    auto nL_of = [&](int j) -> int {
        const int T = GEN ? L - j : span;
        return min(T - 1, max(1, T / 2 - kPairLeftLess128));
    };
    auto nR_of = [&](int j) -> int { return (GEN ? L - j : span) - nL_of(j); };
    const bool has_env = X == 1 && !GEN && N > 1;  // the right tile rebuilds r per sweep (N - 1 steps)
    auto site_of = [&](const PairCur &x) -> int {
        if (x.env) return L - 1 - x.t;
        if (X == 0) return x.j + x.t;
        return GEN ? L - 1 - x.t : (a.R - 1) * N + x.j - x.t;
    };
    auto cur_start = [&]() -> PairCur { return PairCur{0, 0, 0, has_env ? 1 : 0}; };
    auto cur_next = [&](PairCur &x) {
        if (x.env) {
            if (++x.t == N - 1) {
                x.env = 0;
                x.t = 0;
                x.j = 0;
            }
            return;
        }
        if (++x.t == (X == 0 ? nL_of(x.j) : nR_of(x.j))) {
            x.t = 0;
            if (++x.j == N) {
                x.j = 0;
                ++x.sw;
                x.env = has_env ? 1 : 0;
            }
        }
    };
    long long per_sweep = has_env ? N - 1 : 0;
    for (int j = 0; j < N; ++j) per_sweep += X == 0 ? nL_of(j) : nR_of(j);
    const long long total_steps = per_sweep * a.n_sweeps;
    const long long total_atoms = total_steps * C::KA;

    if (warp == 0) tmem_alloc(sa(tmem_slot), 512u);
    if (issuer) {
        for (int s = 0; s < NSG; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(done_bar, 1);
        mbar_init(hand_bar, 1);  // armed by the left with the bytes of one hand-off
        mbar_init(dec_bar, 4);   // one arrival per left epilogue warp
        *abort_flag = 0;
        fence_barrier_init();
        if (X == 0 && total_steps > 0) mbar_expect_tx(hand_bar, HAND_BYTES);  // the first hand-off
    }
    for (int k = tid; k < L; k += SPP_THREADS)
        tab[k] = ((uint32_t)__ldg(GEN ? a.path + k : a.q + (k % N)) & 0xffffu) |
                 ((uint32_t)(__ldg(a.cexp + k) & 0xffff) << 16);
    if (epi) {
        for (int i = 0; i < N; ++i) {
            const uint32_t w = __ballot_sync(FULL, a.spins_in[c * N + i] != 0);
            if (lane == 0) bits[i * 4 + q] = w;
        }
    }
    auto spin = [&](int i) -> int { return (int)((bits[i * 4 + q] >> lane) & 1u); };
    auto site_spin = [&](int k) -> int { return (int)(tab[k] & 0xffffu); };
    auto site_cexp = [&](int k) -> int { return (int)(int16_t)(tab[k] >> 16); };
    auto fail_now = [&]() {
        atomicOr(a.err, 1);
        *abort_flag = 1;
    };
    auto bwait_cluster = [&](uint32_t bar, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (!mbar_wait_cluster(bar, parity, a.wait_limit)) {
            fail_now();
            return false;
        }
        return true;
    };
    // the slice a row takes at the site of x: the proposal's spin flipped
    auto slice_of = [&](const PairCur &x) -> int {
        const int sk = site_spin(site_of(x));
        if (x.env) return spin(sk);
        return spin(sk) ^ (sk == site_spin(x.j) ? 1 : 0);
    };

    // start rows
    int64_t E = 0, El = 0, Ekeep = 0, Eflip = 0;
    double pm = 0.0;
    int64_t pe = 0, acc_count = 0;
    const float *start = X == 0 ? a.bl : a.br;
    if (X == 0) {
        pm = a.state[c].mant;
        pe = a.state[c].exp2;
    } else if (!GEN && active) {
#pragma unroll 1
        for (int ch = 0; ch < CPT; ++ch) {
            float y[64];
            load_chunk(a.br + 64 * ch, y);
            store_chunk(a.rstack + ((size_t)c * a.nr + (a.nr - 1)) * CHI + 64 * ch, y);
        }
        a.rexp[(size_t)c * a.nr + (a.nr - 1)] = 0;
    }
    tc_before();
    cluster_sync_all();  // barriers initialised in both CTAs before any remote arrive
    tc_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tw = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t ta = tw + (uint32_t)C::A_COL;
    const uint32_t tm = tw + (uint32_t)C::META;
    const int lane_a = (lane & 16) | (lane & 7), lane_b = lane_a | 8;
    auto write_meta = [&](const PairCur &x) {
        const int sl = slice_of(x);
        const int s_a = __shfl_sync(FULL, sl, lane_a), s_b = __shfl_sync(FULL, sl, lane_b);
        tmem_st_1(tm, (s_a ? C::HALF1 : C::HALF0) | ((s_b ? C::HALF1 : C::HALF0) << 16));
        if (X == 0 && x.t == 0)  // the first site of a left half-row: the kept slice too
            tmem_st_1(tm + (uint32_t)(C::META2 - C::META),
                      (s_a ? C::HALF0 : C::HALF1) | ((s_b ? C::HALF0 : C::HALF1) << 16));
    };
    auto row_exp = [&](uint32_t col) -> int {
        float m8[8];
#pragma unroll 1
        for (int ch = 0; ch < CPT; ++ch) {
            float y[64];
            tmem_ld_64(tw + col + (uint32_t)(64 * ch), y);
#pragma unroll
            for (int i = 0; i < 64; ++i)
                m8[i & 7] = (ch == 0 && i < 8) ? fabsf(y[i]) : fmaxf(m8[i & 7], fabsf(y[i]));
        }
        const float mx = fmaxf(fmaxf(fmaxf(m8[0], m8[1]), fmaxf(m8[2], m8[3])),
                               fmaxf(fmaxf(m8[4], m8[5]), fmaxf(m8[6], m8[7])));
        const bool usable = (mx > 0.f) && isfinite(mx);
        int e = usable ? rttd::exponent_of(mx) : 0;
        if (__all_sync(FULL, !usable || (e >= 0 && e < 8)) || !usable) e = 0;
        return e;
    };
    auto row_chunk = [&](uint32_t col, int e, int ch, float (&y)[64]) {
        tmem_ld_64(tw + col + (uint32_t)(64 * ch), y);
        scale_chunk(y, e);
    };
    auto write_A_row = [&](const float *src) {
#pragma unroll 1
        for (int ch = 0; ch < CPT; ++ch) {
            float y[64];
            load_chunk(src + 64 * ch, y);
            write_A_chunk<CHI, F16>(ta, ch, y);
        }
    };
    PairCur cur = cur_start();
    if (epi && total_steps > 0) {
        write_A_row(start);
        write_meta(cur);
    }
    tc_before();
    __syncthreads();
    tc_after();

    // producer: atom g = step * KA + at, its own cursor ahead of the steps
    long long g_issued = 0, g_waited = 0;
    PairCur pc = cur_start();
    int p_at = 0;
    auto issue_next = [&]() {
        const long long g = g_issued;
        const int st = (int)(g % NSG);
        const int k = site_of(pc);
        const int y_hi = ((X * 2 + 0) * L + k) * CHI;
        const int y_lo = ((X * 2 + 1) * L + k) * CHI;
        const uint32_t dst = stage0 + (uint32_t)st * C::STAGE;
        mbar_expect_tx(full_bar(st), (uint32_t)C::STAGE);
        tma_load_2d(dst, &map, p_at * 64, y_hi, full_bar(st));
        tma_load_2d(dst + C::BOX, &map, p_at * 64, y_lo, full_bar(st));
        ++g_issued;
        if (++p_at == C::KA) {
            p_at = 0;
            cur_next(pc);
        }
    };
    if (issuer)
        while (g_issued < total_atoms && g_issued < NSG) issue_next();

    const uint32_t peer_dec = peer_addr(dec_bar, 1u);
    const uint32_t peer_hand = peer_addr(hand_bar, 0u);
    const uint32_t peer_buf = peer_addr(sa(hand), 0u);
    long long nhand = 0, ndec = 0;
    int pend = -1;  // right: the spin whose decision is outstanding
    auto settle = [&]() {
        if (pend >= 0) {
            bwait_cluster(dec_bar, (uint32_t)(ndec++ & 1));
            pend = -1;
        }
    };
    bool aborted = false;

    for (long long t = 0; t < total_steps; ++t) {
        const bool dbl = X == 0 && cur.t == 0;
        // ---------------- MMA issue, then the refill (producer)
        if (issuer) {
            const uint32_t a_hi = tmem + (uint32_t)C::A_COL, a_lo = a_hi + (uint32_t)(CHI / 2);
            const uint32_t meta = tmem + (uint32_t)C::META;
            for (int at = 0; at < C::KA; ++at) {
                const long long g = t * C::KA + at;
                const int st = (int)(g % NSG);
                if (!mbar_wait(full_bar(st), (uint32_t)((g / NSG) & 1), a.wait_limit)) {
                    fail_now();
                    break;
                }
                g_waited = g + 1;
                tc_after();
                const uint32_t b_hi = stage0 + (uint32_t)st * C::STAGE, b_lo = b_hi + C::BOX;
                const uint64_t dh0 = sdesc(b_hi), dh1 = sdesc(b_hi + 64);
                const uint64_t dl0 = sdesc(b_lo), dl1 = sdesc(b_lo + 64);
                const uint32_t ao = (uint32_t)(at * 16);
                const uint32_t first = at != 0 ? 1u : 0u;
                mma_sp_ts(tmem, a_hi + ao, dh0, meta, C::IDESC, first);
                mma_sp_ts(tmem, a_hi + ao, dl0, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_lo + ao, dh0, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_hi + ao + 8, dh1, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_hi + ao + 8, dl1, meta, C::IDESC, 1u);
                mma_sp_ts(tmem, a_lo + ao + 8, dh1, meta, C::IDESC, 1u);
                if (dbl) {
                    const uint32_t d2 = tmem + (uint32_t)C::ACC2;
                    const uint32_t meta2 = tmem + (uint32_t)C::META2;
                    mma_sp_ts(d2, a_hi + ao, dh0, meta2, C::IDESC, first);
                    mma_sp_ts(d2, a_hi + ao, dl0, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_lo + ao, dh0, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_hi + ao + 8, dh1, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_hi + ao + 8, dl1, meta2, C::IDESC, 1u);
                    mma_sp_ts(d2, a_lo + ao + 8, dh1, meta2, C::IDESC, 1u);
                }
                mma_commit(empty_bar(st));
            }
            mma_commit(done_bar);
            if (!*abort_flag) {
                for (int at = 0; at < C::KA; ++at) {
                    const long long g = t * C::KA + at;
                    if (g + NSG >= total_atoms) break;
                    const int st = (int)(g % NSG);
                    if (!mbar_wait(empty_bar(st), (uint32_t)((g / NSG) & 1), a.wait_limit)) {
                        fail_now();
                        break;
                    }
                    issue_next();
                }
            }
        }
        bool write_next = false;
        const int k = site_of(cur);
        const int ck = site_cexp(k);
        if (epi && !mbar_wait(done_bar, (uint32_t)(t & 1), a.wait_limit)) fail_now();
        tc_after();
        __syncwarp();
        if (!epi) {
            // the producer warp's other lanes only keep the cursor
        } else if (cur.env) {
            // ---------------- right environment r_k = A_k r_{k+1}
            const int e = row_exp(0u);
            E += e - ck;
            float *dst = a.rstack + ((size_t)c * a.nr + (k - rbase)) * CHI;
            if (active) a.rexp[(size_t)c * a.nr + (k - rbase)] = (int32_t)E;
#pragma unroll 1
            for (int ch = 0; ch < CPT; ++ch) {
                float y[64];
                row_chunk(0u, e, ch, y);
                if (active) store_chunk(dst + 64 * ch, y);
                write_A_chunk<CHI, F16>(ta, ch, y);  // the last one starts proposal 0's half-row
            }
            write_next = true;
        } else if (X == 0) {
            // ---------------- left half-row of proposal j
            const int j = cur.j;
            const bool lastl = cur.t + 1 == nL_of(j);
            int efin;
            if (cur.t == 0) {
                // the kept slice: l_j if the proposal is rejected
                const int e2 = row_exp((uint32_t)C::ACC2);
                Ekeep = El + e2 - ck;
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    row_chunk((uint32_t)C::ACC2, e2, ch, y);
                    if (active) store_chunk(a.lstack + ((size_t)c * N + j) * CHI + 64 * ch, y);
                }
                // the flipped start of the row (l_j if accepted)
                const int e1 = row_exp(0u);
                Eflip = El + e1 - ck;
                E = Eflip;
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    row_chunk(0u, e1, ch, y);
                    if (active) store_chunk(a.tmp + (size_t)c * CHI + 64 * ch, y);
                    if (!lastl) write_A_chunk<CHI, F16>(ta, ch, y);
                }
                efin = e1;
            } else {
                const int e = row_exp(0u);
                E += e - ck;
                if (!lastl) {
#pragma unroll 1
                    for (int ch = 0; ch < CPT; ++ch) {
                        float y[64];
                        row_chunk(0u, e, ch, y);
                        write_A_chunk<CHI, F16>(ta, ch, y);
                    }
                }
                efin = e;
            }
            if (!lastl) {
                write_next = true;
            } else {
                // the right half-row, from the peer CTA; then arm the next hand-off
                bwait_cluster(hand_bar, (uint32_t)(nhand++ & 1));
                const bool next_prop = j + 1 < N;
                const bool next_sweep = !next_prop && cur.sw + 1 < a.n_sweeps;
                if (tid == 0 && (next_prop || next_sweep)) mbar_expect_tx(hand_bar, HAND_BYTES);
                float acc8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    row_chunk(0u, efin, ch, y);
                    dot_hand(y, hand + m * CHI, m, ch, acc8);
                }
                double mm = dot_finish(acc8);
                int64_t Ep = E + hexp[m];
                normalize_scalar(mm, Ep);
                const double ratio = ldexp(mm / pm, (int)(Ep - pe));
                const double x = rttd::mcmc_uniform(a.seed, (uint64_t)(a.chain0 + c),
                                                    (uint64_t)(a.sweep0 + cur.sw), (uint64_t)j);
                const bool accept = active && !*abort_flag && (x < ratio * ratio);
                if (accept) {
                    pm = mm;
                    pe = Ep;
                    ++acc_count;
                    El = Eflip;
                } else {
                    El = Ekeep;
                }
                const int iq = site_spin(j);
                const uint32_t flips = __ballot_sync(FULL, accept);
                if (lane == 0) {
                    const uint32_t w = bits[iq * 4 + q] ^ flips;
                    bits[iq * 4 + q] = w;
                    st_cluster_u32(peer_addr(sa(bits + iq * 4 + q), 1u), w);
                    mbar_arrive_remote(peer_dec);  // the decision is with the right CTA
                }
                __syncwarp();
                // l_j: the flipped start on acceptance (copied over the kept row)
                float *lj = a.lstack + ((size_t)c * N + j) * CHI;
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    load_chunk((accept ? a.tmp + (size_t)c * CHI : lj) + 64 * ch, y);
                    if (accept) store_chunk(lj + 64 * ch, y);
                    if (next_prop) write_A_chunk<CHI, F16>(ta, ch, y);
                }
                if (next_prop) {
                    write_next = true;
                } else if (next_sweep) {
                    write_A_row(a.bl);
                    El = 0;
                    write_next = true;
                }
            }
        } else {
            // ---------------- right half-row of proposal j
            const int j = cur.j;
            const bool lastr = cur.t + 1 == nR_of(j);
            const int e = row_exp(0u);
            E += e - ck;
            if (!lastr) {
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    row_chunk(0u, e, ch, y);
                    write_A_chunk<CHI, F16>(ta, ch, y);
                }
                write_next = true;
            } else {
                settle();  // the previous hand-off has been read
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    row_chunk(0u, e, ch, y);
                    put_hand(y, hand + m * CHI, m, ch);
                }
                hexp[m] = (int32_t)E;
                fence_async_smem();
                bar_sync_n(1, NT);  // the four epilogue warps have written
                if (tid == 0 && !*abort_flag) bulk_copy_to_peer(peer_buf, sa(hand), HAND_BYTES, peer_hand);
                const bool next_prop = j + 1 < N;
                const bool next_sweep = !next_prop && cur.sw + 1 < a.n_sweeps;
                if (next_prop) {  // the next half-row's first MMA does not depend on this decision
                    if (GEN) {
                        write_A_row(a.br);
                        E = 0;
                    } else {
                        write_A_row(a.rstack + ((size_t)c * a.nr + (j + 1)) * CHI);
                        E = a.rexp[(size_t)c * a.nr + (j + 1)];
                    }
                    write_next = true;
                } else if (next_sweep) {
                    write_A_row(a.br);
                    E = 0;
                    write_next = true;
                }
                pend = site_spin(j);  // this proposal's decision is now outstanding
            }
        }
        cur_next(cur);
        if (write_next && epi) {
            if (X == 1 && pend >= 0 && site_spin(site_of(cur)) == pend) settle();
            write_meta(cur);
        }
        tc_before();
        __syncthreads();
        tc_after();
        if (*abort_flag) {
            aborted = true;
            break;
        }
    }
    if (X == 1 && epi) settle();
    // after an expired wait: let a hand-off that is still in flight land
    if (X == 0 && tid == 0 && aborted && total_steps > 0)
        mbar_wait_cluster(hand_bar, (uint32_t)(nhand & 1), a.wait_limit);
    if (X == 0 && !aborted && active) {
        for (int i = 0; i < N; ++i) a.spins_out[c * N + i] = (uint8_t)spin(i);
        a.state[c].mant = pm;
        a.state[c].exp2 = pe;
        if (a.n_accept) a.n_accept[c] += acc_count;
    }
    if (issuer && aborted) {
        for (long long g = g_waited; g < g_issued; ++g)
            mbar_wait(full_bar((int)(g % NSG)), (uint32_t)((g / NSG) & 1), a.wait_limit);
    }
    tc_before();
    cluster_sync_all();  // no CTA leaves while its peer may still store into it
    tc_after();
    if (warp == 0) tmem_dealloc(tmem, 512u);
}


// ------------------------------------------------------------------ flip rows, two tiles per CTA (chi = 128)
// The rows of the local energy with two 128-chain tiles of the same flip row
// j per CTA, so that the epilogue of one tile runs while the tensor pipe
// works on the other (each tile's chain of sites is serial).  Tensor memory
// holds both tiles -- tile u from column 256 u: accumulator [0,128), the hi
// half of the row operand [128,192), metadata at 192 -- because the lo half
// of each row operand lives in shared memory, in 128-byte-swizzled K-major
// atoms that the MMA reads through a descriptor.  Both tiles read the same
// site tensors, streamed once per site by a TMA warp into the ring; a stage
// is released when the second tile's MMAs on it complete.  Warps 0-3:
// epilogue (row m of both tiles), warp 4: MMA issue, warp 5: TMA.  The
// epilogue hands each tile's next operand to the MMA warp through a named
// barrier per tile.
constexpr int R2_THREADS = NT + 64;

// at least 164 KB, so that no other tensor-memory kernel shares the SM
template <int CHI>
inline size_t rows2_smem(int N, int L) {
    return std::max(1024 + (size_t)SCfg<CHI>::NSTG * SCfg<CHI>::STAGE + (size_t)2 * NT * CHI * 2 + 128 +
                        (size_t)32 * N + (size_t)4 * L,
                    (size_t)164 * 1024);
}

// D (+)= A . B with A 2:4 sparse, its compressed entries read from shared
// memory through a descriptor.
__device__ __forceinline__ void mma_sp_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t meta,
                                          uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %5, 0;\n\t"
        "tcgen05.mma.sp.cta_group::1.kind::f16 [%0], %1, %2, [%3], %4, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(meta), "r"(idesc), "r"(accum)
        : "memory");
}
// 32 columns of this warp's 32 TMEM lanes, then wait.
__device__ __forceinline__ void tmem_st_x32(uint32_t t, const uint32_t (&x)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(t), "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]), "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), "r"(x[14]), "r"(x[15]), "r"(x[16]), "r"(x[17]), "r"(x[18]), "r"(x[19]), "r"(x[20]), "r"(x[21]), "r"(x[22]), "r"(x[23]), "r"(x[24]), "r"(x[25]), "r"(x[26]), "r"(x[27]), "r"(x[28]), "r"(x[29]), "r"(x[30]), "r"(x[31])
        : "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

template <int CHI, bool F16>
__global__ void __launch_bounds__(R2_THREADS, 1)
    k_rows2(const __grid_constant__ CUtensorMap map, const Args a) {
    using C = SCfg<CHI, F16>;
    constexpr int NSG = C::NSTG;
    constexpr int CPT = CHI / 64;
    constexpr uint32_t ATOM = (uint32_t)NT * 128;  // one 64-entry K atom of 128 rows
    constexpr uint32_t ALO = CPT * ATOM;           // one tile's lo operand
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t stage0 = sa(base);
    const uint32_t alo0 = stage0 + (uint32_t)(NSG * C::STAGE);
    uint64_t *bars = (uint64_t *)(base + NSG * C::STAGE + 2 * ALO);
    const uint32_t bar0 = sa(bars);
    // bars: full[NSG], empty[NSG], done[2]
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (NSG + s); };
    auto done_bar = [&](int u) { return bar0 + 8u * (2 * NSG + u); };
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NSG + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    long long *issued = (long long *)(bars + 2 * NSG + 3);
    uint32_t *bits = (uint32_t *)((uint8_t *)bars + 128);  // [tile][spin][quadrant]
    uint32_t *tab = bits + 8 * a.N;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool epi = warp < 4;
    const int q = warp & 3;
    const int m = 32 * q + lane;
    const int N = a.N;
    const int j = (int)blockIdx.y;
    int64_t cu[2];
    bool act[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t cr = ((int64_t)blockIdx.x * 2 + u) * NT + m;
        act[u] = epi && cr < a.B;
        cu[u] = cr < a.B ? cr : a.B - 1;
    }
    const long long total_steps = n_steps_of<M_ROWS>(a, j);
    const long long total_atoms = total_steps * C::KA;

    if (warp == 0) tmem_alloc(sa(tmem_slot), 512u);
    if (tid == 0) {
        for (int s = 0; s < NSG; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(done_bar(0), 1);
        mbar_init(done_bar(1), 1);
        *abort_flag = 0;
        issued[0] = 0;
        fence_barrier_init();
    }
    for (int k = tid; k < a.L; k += R2_THREADS)
        tab[k] = ((uint32_t)__ldg(a.path ? a.path + k : a.q + (k % N)) & 0xffffu) |
                 ((uint32_t)(__ldg(a.cexp + k) & 0xffff) << 16);
    if (epi) {
#pragma unroll 1
        for (int u = 0; u < 2; ++u)
            for (int i = 0; i < N; ++i) {
                const uint32_t w = __ballot_sync(FULL, a.spins_in[cu[u] * N + i] != 0);
                if (lane == 0) bits[(u * N + i) * 4 + q] = w;
            }
    }
    auto spin = [&](int u, int i) -> int { return (int)((bits[(u * N + i) * 4 + q] >> lane) & 1u); };
    auto site_spin = [&](int k) -> int { return (int)(tab[k] & 0xffffu); };
    auto site_cexp = [&](int k) -> int { return (int)(int16_t)(tab[k] >> 16); };
    const int iflip = j < N ? (int)(__ldg(a.path ? a.path + j : a.q + j)) : -1;
    auto bwait = [&](uint32_t bar, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (!mbar_wait(bar, parity, a.wait_limit)) {
            atomicOr(a.err, 1);
            *abort_flag = 1;
            return false;
        }
        return true;
    };
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        // ---------------------------------------------------------- MMA issue
        for (long long t = 0; t < total_steps; ++t) {
#pragma unroll 1
            for (int u = 0; u < 2; ++u) {
                named_sync(1 + u, NT + 32);  // tile u's operand for this site is written
                if (lane == 0) {
                    tc_after();
                    const uint32_t d = tmem + 256u * (uint32_t)u;
                    const uint32_t a_hi = d + 128u, meta = d + 192u;
                    const uint32_t a_lo = alo0 + (uint32_t)u * ALO;
                    for (int at = 0; at < C::KA; ++at) {
                        const long long g = t * C::KA + at;
                        const int st = (int)(g % NSG);
                        if (u == 0) bwait(full_bar(st), (uint32_t)((g / NSG) & 1));
                        if (!*abort_flag) {
                            const uint32_t b_hi = stage0 + (uint32_t)st * C::STAGE, b_lo = b_hi + C::BOX;
                            const uint64_t dh0 = sdesc(b_hi), dh1 = sdesc(b_hi + 64);
                            const uint64_t dl0 = sdesc(b_lo), dl1 = sdesc(b_lo + 64);
                            // row entries 32 at .. 32 at + 31: K-steps 2 at and 2 at + 1
                            const uint32_t ao = (uint32_t)(at * 16);
                            const uint64_t al0 = sdesc(a_lo + (uint32_t)(at >> 1) * ATOM + (uint32_t)(at & 1) * 64u);
                            const uint64_t al1 = sdesc(a_lo + (uint32_t)(at >> 1) * ATOM + (uint32_t)(at & 1) * 64u + 32u);
                            const uint32_t first = at != 0 ? 1u : 0u;
                            mma_sp_ts(d, a_hi + ao, dh0, meta, C::IDESC, first);
                            mma_sp_ts(d, a_hi + ao, dl0, meta, C::IDESC, 1u);
                            mma_sp_ss(d, al0, dh0, meta, C::IDESC, 1u);
                            mma_sp_ts(d, a_hi + ao + 8, dh1, meta, C::IDESC, 1u);
                            mma_sp_ts(d, a_hi + ao + 8, dl1, meta, C::IDESC, 1u);
                            mma_sp_ss(d, al1, dh1, meta, C::IDESC, 1u);
                        }
                        if (u == 1) mma_commit(empty_bar(st));  // both tiles have read the stage
                    }
                    mma_commit(done_bar(u));
                }
                __syncwarp();
            }
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------- TMA
        if (lane == 0) {
            for (long long g = 0; g < total_atoms; ++g) {
                const int st = (int)(g % NSG);
                if (g >= NSG && !bwait(empty_bar(st), (uint32_t)(((g / NSG) - 1) & 1))) break;
                if (*abort_flag) break;
                const int k = j + (int)(g / C::KA), at = (int)(g % C::KA);
                const uint32_t dst = stage0 + (uint32_t)st * C::STAGE;
                mbar_expect_tx(full_bar(st), (uint32_t)C::STAGE);
                tma_load_2d(dst, &map, at * 64, (0 * a.L + k) * CHI, full_bar(st));
                tma_load_2d(dst + C::BOX, &map, at * 64, (1 * a.L + k) * CHI, full_bar(st));
                issued[0] = g + 1;
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue (rows m of both tiles)
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        const int lane_a = (lane & 16) | (lane & 7), lane_b = lane_a | 8;
        auto write_meta = [&](int u, int k) {
            const int sk = site_spin(k);
            const int sl = spin(u, sk) ^ (sk == iflip ? 1 : 0);
            const int s_a = __shfl_sync(FULL, sl, lane_a), s_b = __shfl_sync(FULL, sl, lane_b);
            tmem_st_1(tq + 256u * (uint32_t)u + 192u,
                      (s_a ? C::HALF1 : C::HALF0) | ((s_b ? C::HALF1 : C::HALF0) << 16));
        };
        // entries 64 ch .. 64 ch + 63 of row m as tile u's operand: hi into
        // TMEM, lo into the swizzled shared-memory atom ch
        auto write_op = [&](int u, int ch, const float (&y)[64]) {
            uint32_t hh[32], ll[32];
#pragma unroll
            for (int p = 0; p < 32; ++p) split2<F16>(y[2 * p], y[2 * p + 1], hh[p], ll[p]);
            tmem_st_x32(tq + 256u * (uint32_t)u + 128u + (uint32_t)(32 * ch), hh);
            const uint32_t row = alo0 + (uint32_t)u * ALO + (uint32_t)ch * ATOM + (uint32_t)m * 128u;
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8)
                st_shared_v4(row + ((uint32_t)(c8 ^ (m & 7)) << 4), ll[4 * c8], ll[4 * c8 + 1],
                             ll[4 * c8 + 2], ll[4 * c8 + 3]);
        };
        auto publish = [&](int u) {
            fence_async_smem();
            tc_before();
            named_arrive(1 + u, NT + 32);
        };
        auto row_exp = [&](int u) -> int {
            float m8[8];
#pragma unroll 1
            for (int ch = 0; ch < CPT; ++ch) {
                float y[64];
                tmem_ld_64(tq + 256u * (uint32_t)u + (uint32_t)(64 * ch), y);
#pragma unroll
                for (int i = 0; i < 64; ++i)
                    m8[i & 7] = (ch == 0 && i < 8) ? fabsf(y[i]) : fmaxf(m8[i & 7], fabsf(y[i]));
            }
            const float mx = fmaxf(fmaxf(fmaxf(m8[0], m8[1]), fmaxf(m8[2], m8[3])),
                                   fmaxf(fmaxf(m8[4], m8[5]), fmaxf(m8[6], m8[7])));
            const bool usable = (mx > 0.f) && isfinite(mx);
            int e = usable ? rttd::exponent_of(mx) : 0;
            if (__all_sync(FULL, !usable || (e >= 0 && e < 8)) || !usable) e = 0;
            return e;
        };
        int64_t E[2] = {0, 0}, fin_E[2] = {0, 0};
        double fin_m[2] = {0.0, 0.0};
        const float *start[2] = {a.bl, a.bl};
        if (j > 0) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                start[u] = a.lstack + ((size_t)cu[u] * N + (j - 1)) * CHI;
                E[u] = a.lexp[(size_t)cu[u] * N + (j - 1)];
            }
        }
        const int rq = row_end(a, j) + 1 - a.kmin;  // r_{end+1}; b_R for j = N
        if (total_steps > 0) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    load_chunk(start[u] + 64 * ch, y);
                    write_op(u, ch, y);
                }
                write_meta(u, j);
                publish(u);
            }
        }
        for (long long t = 0; t < total_steps; ++t) {
            const int k = j + (int)t;
            const int ck = site_cexp(k);
            const bool last = t + 1 == total_steps;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                bwait(done_bar(u), (uint32_t)(t & 1));
                tc_after();
                __syncwarp();
                const int e = row_exp(u);
                E[u] += e - ck;
                if (!last) {
#pragma unroll 1
                    for (int ch = 0; ch < CPT; ++ch) {
                        float y[64];
                        tmem_ld_64(tq + 256u * (uint32_t)u + (uint32_t)(64 * ch), y);
                        scale_chunk(y, e);
                        write_op(u, ch, y);
                    }
                    write_meta(u, k + 1);
                    publish(u);
                } else {
                    const float *rclose = a.rstack + ((size_t)cu[u] * a.nr + rq) * CHI;
                    float acc8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
                    for (int ch = 0; ch < CPT; ++ch) {
                        float y[64];
                        tmem_ld_64(tq + 256u * (uint32_t)u + (uint32_t)(64 * ch), y);
                        scale_chunk(y, e);
                        dot_chunk(y, rclose + 64 * ch, acc8);
                    }
                    fin_m[u] = dot_finish(acc8);
                    fin_E[u] = E[u] + a.rexp[(size_t)cu[u] * a.nr + rq];
                }
            }
        }
        if (total_steps == 0) {
            // no site steps (R = 1 and the unflipped row in the first block):
            // the start row closes on r_{end+1}
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float *rclose = a.rstack + ((size_t)cu[u] * a.nr + rq) * CHI;
                float acc8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
                for (int ch = 0; ch < CPT; ++ch) {
                    float y[64];
                    load_chunk(start[u] + 64 * ch, y);
                    dot_chunk(y, rclose + 64 * ch, acc8);
                }
                fin_m[u] = dot_finish(acc8);
                fin_E[u] = E[u] + a.rexp[(size_t)cu[u] * a.nr + rq];
            }
        }
        if (!*abort_flag) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (act[u]) {
                    double mm = fin_m[u];
                    int64_t Ep = fin_E[u];
                    normalize_scalar(mm, Ep);
                    a.rows_mant[cu[u] * (N + 1) + j] = mm;
                    a.rows_exp[cu[u] * (N + 1) + j] = Ep;
                }
        }
    }
    // ---------------- teardown: drain own copies (bounded), free TMEM
    tc_before();
    __syncthreads();
    tc_after();
    if (tid == 5 * 32 && *abort_flag) {
        const long long n = issued[0];
        for (long long g = (n > NSG ? n - NSG : 0); g < n; ++g)
            mbar_wait(full_bar((int)(g % NSG)), (uint32_t)((g / NSG) & 1), a.wait_limit);
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512u);
}

}  // namespace tcd

// ====================================================================== host side
void *tc_encode_tiled_fn() {
    static void *fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = p;
    }
    return fn;
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    return (EncodeTiledFn)tc_encode_tiled_fn();
}

inline void split16(double x, bool f16, uint16_t &hi, uint16_t &lo) {
    const float xf = (float)x;
    if (f16) {
        const __half h = __float2half_rn(xf);
        const __half l = __float2half_rn(xf - __half2float(h));
        hi = *reinterpret_cast<const uint16_t *>(&h);
        lo = *reinterpret_cast<const uint16_t *>(&l);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(xf);
        const __nv_bfloat16 l = __float2bfloat16_rn(xf - __bfloat162float(h));
        hi = *reinterpret_cast<const uint16_t *>(&h);
        lo = *reinterpret_cast<const uint16_t *>(&l);
    }
}

tcd::Args make_args(rtt_s *h, int64_t B) {
    tcd::Args a;
    memset(&a, 0, sizeof(a));
    TcPlan *p = h->tc;
    a.bl = p->d_bl;
    a.br = p->d_br;
    a.q = h->d_q;
    a.cexp = p->d_cexp;
    a.N = h->N;
    a.L = h->L;
    a.R = h->R;
    a.B = B;
    a.lstack = (float *)h->d_lstack;
    a.lexp = h->d_lexp;
    a.rstack = (float *)h->d_rstack;
    a.rexp = h->d_rexp;
    a.rows_mant = h->d_rows_mant;
    a.rows_exp = h->d_rows_exp;
    a.path = h->periodic ? nullptr : h->d_path;
    a.last = h->d_last;
    a.kmin = h->kmin;
    a.nr = h->nr;
    a.err = p->d_err;
    a.wait_limit = 4000000000LL;  // ~2 s at 2 GHz
    return a;
}

template <int CHI, int MODE, bool F16>
cudaError_t launch(const TcPlan *p, const tcd::Args &a, dim3 grid, cudaStream_t st) {
    const size_t smem = tcd::SCfg<CHI, F16>::smem_bytes(a.N, a.L);
    cudaError_t e = cudaFuncSetAttribute(tcd::k_tc<CHI, MODE, F16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tcd::k_tc<CHI, MODE, F16><<<grid, tcd::NT * tcd::SCfg<CHI, F16>::NH + 32, smem, st>>>(p->map_sp, a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_chi(const TcPlan *p, const tcd::Args &a, dim3 grid, cudaStream_t st) {
    if (p->chi == 64) return p->f16 ? launch<64, MODE, true>(p, a, grid, st)
                                    : launch<64, MODE, false>(p, a, grid, st);
    if (p->chi == 128) return p->f16 ? launch<128, MODE, true>(p, a, grid, st)
                                     : launch<128, MODE, false>(p, a, grid, st);
    return cudaErrorInvalidValue;
}

rtt_status status_of(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return RTT_OK;
    rtt_set_error(std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? RTT_ERR_OOM : RTT_ERR_CUDA;
}

unsigned tiles(int64_t B) { return (unsigned)((B + tcd::NT - 1) / tcd::NT); }

}  // namespace

rtt_status tc_plan_create(rtt_s *h, const double *tensors, const double *bl, const double *br) {
    const int chi = h->chi, L = h->L;
    if (!tc_supported_chi(chi) || h->chip != chi) {
        rtt_set_error("BF16X3 / FP16X3 support chi in {64, 128}");
        return RTT_ERR_UNSUPPORTED;
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        rtt_set_error("cuTensorMapEncodeTiled unavailable from the driver");
        return RTT_ERR_CUDA;
    }
    TcPlan *p = new TcPlan();
    h->tc = p;
    p->chi = chi;
    p->f16 = (h->precision == RTT_FP16X3);
    // exact per-site prescale 2^c_k bringing max|A_k| into [1,2)
    std::vector<int32_t> cexp(L, 0);
    for (int k = 0; k < L; ++k) {
        double mx = 0.0;
        for (size_t i = 0; i < (size_t)2 * chi * chi; ++i)
            mx = std::max(mx, std::fabs(tensors[(size_t)k * 2 * chi * chi + i]));
        cexp[k] = (mx > 0.0) ? -std::ilogb(mx) : 0;
    }
    cudaError_t e;
    // sparse operand of the generic tile kernel: row n, K index 2x + s
    {
        const size_t rows = (size_t)4 * L * chi, K = (size_t)2 * chi;
        std::vector<uint16_t> Bs(rows * K);
        for (int k = 0; k < L; ++k)
            for (int s = 0; s < 2; ++s) {
                const double *A = tensors + ((size_t)k * 2 + s) * chi * chi;
                for (int n = 0; n < chi; ++n)
                    for (int x = 0; x < chi; ++x) {
                        // left to right: output b = n, contracted a = x
                        const double xt = std::ldexp(A[(size_t)x * chi + n], cexp[k]);
                        // right to left: output a = n, contracted b = x
                        const double xb = std::ldexp(A[(size_t)n * chi + x], cexp[k]);
                        const size_t col = (size_t)2 * x + s;
                        split16(xt, p->f16, Bs[((size_t)(0 * L + k) * chi + n) * K + col],
                                Bs[((size_t)(1 * L + k) * chi + n) * K + col]);
                        split16(xb, p->f16, Bs[((size_t)(2 * L + k) * chi + n) * K + col],
                                Bs[((size_t)(3 * L + k) * chi + n) * K + col]);
                    }
            }
        if ((e = cudaMalloc((void **)&p->d_Bs, Bs.size() * sizeof(uint16_t))) != cudaSuccess)
            return status_of(e, "tc plan: tensors");
        if ((e = cudaMemcpy(p->d_Bs, Bs.data(), Bs.size() * sizeof(uint16_t),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return status_of(e, "tc plan: tensors copy");
        const cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
        const cuuint64_t gstride[1] = {(cuuint64_t)K * sizeof(uint16_t)};
        const cuuint32_t box[2] = {64u, (cuuint32_t)chi};
        const cuuint32_t estride[2] = {1u, 1u};
        CUresult r = enc(&p->map_sp,
                         p->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                         2, p->d_Bs, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            rtt_set_error("cuTensorMapEncodeTiled failed (sparse operand)");
            return RTT_ERR_CUDA;
        }
    }
    // dense operand of the chi = 64 split-row sweep
    if (chi == 64) {
        const size_t rows = (size_t)4 * L * 2 * chi;
        std::vector<uint16_t> Bh(rows * chi);
        for (int k = 0; k < L; ++k)
            for (int s = 0; s < 2; ++s)
                for (int n = 0; n < chi; ++n)
                    for (int kk = 0; kk < chi; ++kk) {
                        const double *A = tensors + ((size_t)k * 2 + s) * chi * chi;
                        // left-to-right operand: row n = output column b, K index = a
                        const double xt = std::ldexp(A[(size_t)kk * chi + n], cexp[k]);
                        // right-to-left operand: row n = output index a, K index = b
                        const double xb = std::ldexp(A[(size_t)n * chi + kk], cexp[k]);
                        const size_t r0 = ((size_t)(0 * L + k) * 2 * chi + s * chi + n) * chi + kk;
                        const size_t r1 = ((size_t)(1 * L + k) * 2 * chi + s * chi + n) * chi + kk;
                        const size_t r2 = ((size_t)(2 * L + k) * 2 * chi + s * chi + n) * chi + kk;
                        const size_t r3 = ((size_t)(3 * L + k) * 2 * chi + s * chi + n) * chi + kk;
                        split16(xt, p->f16, Bh[r0], Bh[r1]);
                        split16(xb, p->f16, Bh[r2], Bh[r3]);
                    }
        if ((e = cudaMalloc((void **)&p->d_B, Bh.size() * sizeof(uint16_t))) != cudaSuccess)
            return status_of(e, "tc plan: tensors");
        if ((e = cudaMemcpy(p->d_B, Bh.data(), Bh.size() * sizeof(uint16_t),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return status_of(e, "tc plan: tensors copy");
        const cuuint64_t gdim[2] = {(cuuint64_t)chi, (cuuint64_t)rows};
        const cuuint64_t gstride[1] = {(cuuint64_t)chi * sizeof(uint16_t)};
        const cuuint32_t box[2] = {64u, (cuuint32_t)(2 * chi)};
        const cuuint32_t estride[2] = {1u, 1u};
        CUresult r = enc(&p->map,
                         p->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                         2, p->d_B, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            rtt_set_error("cuTensorMapEncodeTiled failed");
            return RTT_ERR_CUDA;
        }
    }
    if ((e = cudaMalloc((void **)&p->d_cexp, (size_t)L * sizeof(int32_t))) != cudaSuccess)
        return status_of(e, "tc plan: prescale");
    cudaMemcpy(p->d_cexp, cexp.data(), (size_t)L * sizeof(int32_t), cudaMemcpyHostToDevice);
    std::vector<float> blf(chi), brf(chi);
    for (int i = 0; i < chi; ++i) {
        blf[i] = (float)bl[i];
        brf[i] = (float)br[i];
    }
    if ((e = cudaMalloc((void **)&p->d_bl, chi * 4)) != cudaSuccess) return status_of(e, "tc plan");
    if ((e = cudaMalloc((void **)&p->d_br, chi * 4)) != cudaSuccess) return status_of(e, "tc plan");
    cudaMemcpy(p->d_bl, blf.data(), chi * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_br, brf.data(), chi * 4, cudaMemcpyHostToDevice);
    if ((e = cudaMalloc((void **)&p->d_err, sizeof(int))) != cudaSuccess) return status_of(e, "tc plan");
    cudaMemset(p->d_err, 0, sizeof(int));
    return RTT_OK;
}

void tc_plan_destroy(rtt_s *h) {
    TcPlan *p = h->tc;
    if (!p) return;
    cudaFree(p->d_B);
    cudaFree(p->d_Bs);
    cudaFree(p->d_cexp);
    cudaFree(p->d_bl);
    cudaFree(p->d_br);
    cudaFree(p->d_tmp);
    cudaFree(p->d_tmp_exp);
    cudaFree(p->d_err);
    delete p;
    h->tc = nullptr;
}

rtt_status tc_left_env(rtt_s *h, const uint8_t *spins, int64_t B, cudaStream_t st) {
    tcd::Args a = make_args(h, B);
    a.spins_in = spins;
    prof_begin(h, KID_TC_LEFT_ENV, st);
    cudaError_t e = launch_chi<tcd::M_LEFT>(h->tc, a, dim3(tiles(B)), st);
    prof_end(h, KID_TC_LEFT_ENV, st);
    return status_of(e, "tc left environments");
}

rtt_status tc_right_env(rtt_s *h, const uint8_t *spins, int64_t B, cudaStream_t st) {
    tcd::Args a = make_args(h, B);
    a.spins_in = spins;
    prof_begin(h, KID_TC_RIGHT_ENV, st);
    cudaError_t e = launch_chi<tcd::M_RIGHT>(h->tc, a, dim3(tiles(B)), st);
    prof_end(h, KID_TC_RIGHT_ENV, st);
    return status_of(e, "tc right environments");
}

rtt_status tc_rows(rtt_s *h, const uint8_t *spins, int64_t B, cudaStream_t st) {
    tcd::Args a = make_args(h, B);
    a.spins_in = spins;
    prof_begin(h, KID_TC_ROWS, st);
    cudaError_t e;
    const size_t smem2 = h->tc->chi == 128 ? tcd::rows2_smem<128>(h->N, h->L) : tcd::rows2_smem<64>(h->N, h->L);
    if (smem2 <= (size_t)227 * 1024) {
        // two tiles per CTA (one tile's epilogue beside the other's MMAs)
        auto go = [&](auto kern) {
            cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
            if (err == cudaSuccess)
                kern<<<dim3((tiles(B) + 1) / 2, h->N + 1), tcd::R2_THREADS, smem2, st>>>(h->tc->map_sp, a);
            return err;
        };
        if (h->tc->chi == 128)
            e = h->tc->f16 ? go(tcd::k_rows2<128, true>) : go(tcd::k_rows2<128, false>);
        else
            e = h->tc->f16 ? go(tcd::k_rows2<64, true>) : go(tcd::k_rows2<64, false>);
        if (e == cudaSuccess) e = cudaGetLastError();
    } else {
        e = launch_chi<tcd::M_ROWS>(h->tc, a, dim3(tiles(B), h->N + 1), st);
    }
    prof_end(h, KID_TC_ROWS, st);
    return status_of(e, "tc flip rows");
}

rtt_status tc_chain_init(rtt_s *h, const uint8_t *spins, int64_t B, double *log_abs, int8_t *sign,
                         rtt_chain_state *state, cudaStream_t st) {
    tcd::Args a = make_args(h, B);
    a.spins_in = spins;
    a.log_abs = log_abs;
    a.sign = sign;
    a.state = state;
    prof_begin(h, KID_TC_CHAIN_INIT, st);
    cudaError_t e = launch_chi<tcd::M_INIT>(h->tc, a, dim3(tiles(B)), st);
    prof_end(h, KID_TC_CHAIN_INIT, st);
    return status_of(e, "tc log amplitudes");
}

rtt_status tc_sweep(rtt_s *h, uint8_t *spins, rtt_chain_state *state, int64_t B, int64_t chain0,
                    int64_t sweep0, int32_t n_sweeps, int64_t *n_accept, cudaStream_t st) {
    TcPlan *p = h->tc;
    if (B > p->tmp_cap) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return status_of(e, "tc sweep scratch");
        cudaFree(p->d_tmp);
        cudaFree(p->d_tmp_exp);
        p->d_tmp = nullptr;
        p->d_tmp_exp = nullptr;
        p->tmp_cap = 0;
        // [2][B][chi]: flipped row starts, then right half-rows of the split sweep
        if ((e = cudaMalloc((void **)&p->d_tmp, (size_t)2 * B * p->chi * 4)) != cudaSuccess)
            return status_of(e, "tc sweep scratch");
        if ((e = cudaMalloc((void **)&p->d_tmp_exp, (size_t)2 * B * 4)) != cudaSuccess)
            return status_of(e, "tc sweep scratch");
        p->tmp_cap = B;
    }
    tcd::Args a = make_args(h, B);
    a.lstack = (float *)h->d_sw_lstack;
    a.lexp = h->d_sw_lexp;
    a.rstack = (float *)h->d_sw_rstack;
    a.rexp = h->d_sw_rexp;
    a.spins_in = spins;
    a.spins_out = spins;
    a.state = state;
    a.tmp = p->d_tmp;
    a.tmp_exp = p->d_tmp_exp;
    a.chain0 = chain0;
    a.sweep0 = sweep0;
    a.n_sweeps = n_sweeps;
    a.seed = h->seed;
    a.n_accept = n_accept;
    cudaError_t e;
    prof_begin(h, KID_TC_SWEEP, st);
    const size_t smem_pair128 = std::max(tcd::spp_smem(h->N, h->L), (size_t)164 * 1024);
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const bool pair128 = p->chi == 128 && h->R >= 2 && h->N >= 2 && smem_pair128 <= (size_t)227 * 1024 &&
                         2 * (int64_t)tiles(B) <= (int64_t)n_sm;
    if (!h->periodic && !(p->chi == 64 && h->R >= 2 && h->N >= 2) && !pair128) {
        prof_end(h, KID_TC_SWEEP, st);
        rtt_set_error("rtt_mcmc_sweep: tensor-core sweeps on a general path need at least two "
                      "replicas, and at chi = 128 a batch whose CTA pairs fit on the GPU at once");
        return RTT_ERR_UNSUPPORTED;
    }
    if (pair128) {
        // split-row sweep on CTA pairs with the sparse site products, while the
        // pairs fit on the GPU at once (measured: 64 tiles of 16x16 chains run
        // 1.8x faster than on single tiles; 128 tiles of 10x10 chains, two
        // waves of pairs, 11 % slower); the same shared-memory floor keeps
        // every other TMEM-allocating CTA off its SMs
        auto go = [&](auto kern) {
            cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem_pair128);
            if (err == cudaSuccess) kern<<<2 * tiles(B), tcd::SPP_THREADS, smem_pair128, st>>>(p->map_sp, a);
            return err;
        };
        if (h->periodic)
            e = p->f16 ? go(tcd::k_sp_pair<true, false>) : go(tcd::k_sp_pair<false, false>);
        else
            e = p->f16 ? go(tcd::k_sp_pair<true, true>) : go(tcd::k_sp_pair<false, true>);
        if (e == cudaSuccess) e = cudaGetLastError();
    } else if (p->chi == 64 && h->R >= 2 && h->N >= 2) {
        // split-row sweep on CTA pairs.  At least 164 KB of shared memory: no
        // other CTA that allocates TMEM (a second pair CTA, a 66 KB tile kernel
        // of the energy) fits beside a pair CTA on one SM, so no tcgen05.alloc
        // ever waits for a CTA that waits for its cluster peer
        const size_t smemc = std::max(tcd::sweepc_smem(h->N, h->L), (size_t)164 * 1024);
        auto goc = [&](auto kern) {
            cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smemc);
            if (err == cudaSuccess) kern<<<2 * tiles(B), tcd::SPC_THREADS, smemc, st>>>(p->map, a);
            return err;
        };
        if (h->periodic)
            e = p->f16 ? goc(tcd::k_tc_sweep_pair<true, false>) : goc(tcd::k_tc_sweep_pair<false, false>);
        else
            e = p->f16 ? goc(tcd::k_tc_sweep_pair<true, true>) : goc(tcd::k_tc_sweep_pair<false, true>);
        if (e == cudaSuccess) e = cudaGetLastError();
    } else {
        e = launch_chi<tcd::M_SWEEP>(p, a, dim3(tiles(B)), st);
    }
    prof_end(h, KID_TC_SWEEP, st);
    return status_of(e, "tc sweep");
}

int *tc_error_word(rtt_s *h) { return h->tc ? h->tc->d_err : nullptr; }

rtt_status tc_wait_selftest(rtt_s *h, long long budget_cycles, cudaStream_t st) {
    tcd::k_wait_selftest<<<1, 32, 0, st>>>(h->tc->d_err, budget_cycles);
    return status_of(cudaGetLastError(), "wait self-test");
}
