// rtt_tc.cu -- tensor-core form of the RTT site chain (sm_103a, tcgen05).
//
// Per site k the rows of a 128-chain tile are contracted with both spin
// slices at once, D[128 x 2chi] = V[128 x chi] . [A_k[0] | A_k[1]] (Eq. RTT
// evaluated left to right; right-to-left steps use the transposed slices),
// on the 5th-generation tensor cores:
//   - operands in 16-bit hi/lo split form, x = hi + lo + O(u^2 |x|) with u
//     the unit roundoff of the 16-bit type (BF16: 2^-8, FP16: 2^-11); three
//     products hi.hi + hi.lo + lo.hi accumulate in FP32 in TMEM.  Each site
//     tensor is prescaled by an exact power of two 2^c_k (max entry in [1,2))
//     so that FP16 stays in its normal range; c_k is taken back out of the
//     integer exponent sum;
//   - the site tensors are streamed by TMA (128-byte swizzle, K-major) into a
//     two-stage shared-memory ring; the rows live in shared memory in the
//     same swizzled K-major layout, written by the epilogue;
//   - epilogue (one thread per row = TMEM lane): load both accumulator
//     halves, keep the half of the row's spin at site k, rescale by an exact
//     power of two (exponent summed in an integer), split to hi/lo BF16 and
//     store the row back as the next site's A operand.
// Thread 0 issues TMA and MMA; every wait is bounded by a clock budget after
// which the CTA records an error flag, drains its own copies, frees its TMEM
// and returns.
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
    uint16_t *d_B = nullptr;       // [4][L][2chi][chi]: BT hi, BT lo, B hi, B lo
    int32_t *d_cexp = nullptr;     // [L] prescale exponents c_k
    float *d_bl = nullptr, *d_br = nullptr;
    CUtensorMap map;
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
    static constexpr int A_ATOM = 128 * 128;       // bytes: 128 rows x 128 B
    static constexpr int A_BYTES = KA * A_ATOM;    // one of hi / lo
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
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

// Two 64-column loads (32x32b.x64) -- the same column block of both
// accumulator halves -- and the wait, in one statement.
__device__ __forceinline__ void tmem_ld_2x64(uint32_t t0, uint32_t t1, uint32_t (&x)[64],
                                             uint32_t (&y)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%128];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79,"
        "%80,%81,%82,%83,%84,%85,%86,%87,%88,%89,%90,%91,%92,%93,%94,%95,"
        "%96,%97,%98,%99,%100,%101,%102,%103,%104,%105,%106,%107,%108,%109,%110,%111,"
        "%112,%113,%114,%115,%116,%117,%118,%119,%120,%121,%122,%123,%124,%125,%126,%127}, [%129];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]),
          "=r"(x[7]), "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]),
          "=r"(x[13]), "=r"(x[14]), "=r"(x[15]), "=r"(x[16]), "=r"(x[17]), "=r"(x[18]),
          "=r"(x[19]), "=r"(x[20]), "=r"(x[21]), "=r"(x[22]), "=r"(x[23]), "=r"(x[24]),
          "=r"(x[25]), "=r"(x[26]), "=r"(x[27]), "=r"(x[28]), "=r"(x[29]), "=r"(x[30]),
          "=r"(x[31]), "=r"(x[32]), "=r"(x[33]), "=r"(x[34]), "=r"(x[35]), "=r"(x[36]),
          "=r"(x[37]), "=r"(x[38]), "=r"(x[39]), "=r"(x[40]), "=r"(x[41]), "=r"(x[42]),
          "=r"(x[43]), "=r"(x[44]), "=r"(x[45]), "=r"(x[46]), "=r"(x[47]), "=r"(x[48]),
          "=r"(x[49]), "=r"(x[50]), "=r"(x[51]), "=r"(x[52]), "=r"(x[53]), "=r"(x[54]),
          "=r"(x[55]), "=r"(x[56]), "=r"(x[57]), "=r"(x[58]), "=r"(x[59]), "=r"(x[60]),
          "=r"(x[61]), "=r"(x[62]), "=r"(x[63]), "=r"(y[0]), "=r"(y[1]), "=r"(y[2]),
          "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7]), "=r"(y[8]), "=r"(y[9]),
          "=r"(y[10]), "=r"(y[11]), "=r"(y[12]), "=r"(y[13]), "=r"(y[14]), "=r"(y[15]),
          "=r"(y[16]), "=r"(y[17]), "=r"(y[18]), "=r"(y[19]), "=r"(y[20]), "=r"(y[21]),
          "=r"(y[22]), "=r"(y[23]), "=r"(y[24]), "=r"(y[25]), "=r"(y[26]), "=r"(y[27]),
          "=r"(y[28]), "=r"(y[29]), "=r"(y[30]), "=r"(y[31]), "=r"(y[32]), "=r"(y[33]),
          "=r"(y[34]), "=r"(y[35]), "=r"(y[36]), "=r"(y[37]), "=r"(y[38]), "=r"(y[39]),
          "=r"(y[40]), "=r"(y[41]), "=r"(y[42]), "=r"(y[43]), "=r"(y[44]), "=r"(y[45]),
          "=r"(y[46]), "=r"(y[47]), "=r"(y[48]), "=r"(y[49]), "=r"(y[50]), "=r"(y[51]),
          "=r"(y[52]), "=r"(y[53]), "=r"(y[54]), "=r"(y[55]), "=r"(y[56]), "=r"(y[57]),
          "=r"(y[58]), "=r"(y[59]), "=r"(y[60]), "=r"(y[61]), "=r"(y[62]), "=r"(y[63])
        : "r"(t0), "r"(t1)
        : "memory");
}

// ------------------------------------------------------------------ row helpers
// Accumulator half `sel` (0: columns [0,chi), 1: [chi,2chi)) of this thread's
// TMEM lane.  The column address of tcgen05.ld is warp-uniform, so both halves
// are loaded and the row's half is selected in registers.
template <int CHI>
__device__ __forceinline__ void acc_select(uint32_t tw, int sel, float (&v)[CHI]) {
    if constexpr (CHI == 64) {
        uint32_t x0[64], x1[64];
        tmem_ld_2x64(tw, tw + CHI, x0, x1);
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(sel ? x1[i] : x0[i]);
    } else {
#pragma unroll
        for (int c = 0; c < CHI; c += 32) {
            uint32_t x0[32], x1[32];
            tmem_ld_2x32(tw + c, tw + CHI + c, x0, x1);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[c + i] = __uint_as_float(sel ? x1[i] : x0[i]);
        }
    }
}

// Rescale by an exact power of two so that max|v| lies in [1,2) (or leave
// the row alone while max|v| is in [1, 2^8), see below); returns the exponent
// taken out.  Eight independent partial maxima keep the dependency chain short.
template <int CHI, bool LAZY = true>
__device__ __forceinline__ int renorm(float (&v)[CHI]) {
    float m[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) m[p] = fabsf(v[p]);
#pragma unroll
    for (int i = 8; i < CHI; ++i) m[i & 7] = fmaxf(m[i & 7], fabsf(v[i]));
    const float mx = fmaxf(fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3])),
                           fmaxf(fmaxf(m[4], m[5]), fmaxf(m[6], m[7])));
    const bool usable = (mx > 0.f) && isfinite(mx);
    const int e = usable ? rttd::exponent_of(mx) : 0;
    // A row whose max lies in [1, 2^8) can keep its scale: its 16-bit split is
    // inside FP16's normal range with full precision relative to the max, and
    // the next site's accumulator (FP32) is rescaled again before its split
    // unless it too lands in the window.  The warp skips the rescale when all
    // of its rows can (all lanes of the warp call this together).
    if (LAZY && __all_sync(FULL, !usable || (e >= 0 && e < 8))) return 0;
    if (!usable) return 0;
    if (rttd::pow2_normal(0.f, -e)) {  // one exact multiply per entry
        const float sc = rttd::pow2(0.f, -e);
#pragma unroll
        for (int i = 0; i < CHI; ++i) v[i] *= sc;
    } else {
#pragma unroll
        for (int i = 0; i < CHI; ++i) v[i] = rttd::scale2(v[i], -e);
    }
    return e;
}

// Split the row into 16-bit hi/lo and store it as row m of the A operand
// (K-major, 128-byte swizzle: 16-byte chunk c of row m sits at c ^ (m & 7)).
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

template <int CHI, bool F16>
__device__ __forceinline__ void write_A(uint32_t a_hi, uint32_t a_lo, int m, const float (&v)[CHI]) {
#pragma unroll
    for (int at = 0; at < CHI / 64; ++at) {
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int p = 0; p < 4; ++p)
                split2<F16>(v[at * 64 + ch * 8 + 2 * p], v[at * 64 + ch * 8 + 2 * p + 1], h[p], l[p]);
            const uint32_t off =
                (uint32_t)(at * Cfg<CHI>::A_ATOM + m * 128 + ((ch ^ (m & 7)) << 4));
            st_shared_v4(a_hi + off, h[0], h[1], h[2], h[3]);
            st_shared_v4(a_lo + off, l[0], l[1], l[2], l[3]);
        }
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
// Closing contraction sum_b v_b r_b: eight FP32 partial sums (fma), combined
// in FP64.
template <int CHI>
__device__ __forceinline__ double dot(const float (&v)[CHI], const float *__restrict__ r) {
    float acc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) acc[p] = 0.f;
    const float4 *r4 = reinterpret_cast<const float4 *>(r);
#pragma unroll
    for (int i = 0; i < CHI / 4; ++i) {
        const float4 x = r4[i];
        const int p = (2 * i) & 7;
        acc[p] = fmaf(v[4 * i], x.x, acc[p]);
        acc[p + 1] = fmaf(v[4 * i + 1], x.y, acc[p + 1]);
        acc[(p + 2) & 7] = fmaf(v[4 * i + 2], x.z, acc[(p + 2) & 7]);
        acc[(p + 3) & 7] = fmaf(v[4 * i + 3], x.w, acc[(p + 3) & 7]);
    }
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < 8; ++p) s += (double)acc[p];
    return s;
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
// Row m of the A operand in TMEM: the 16-bit hi/lo split of v, entries 2c and
// 2c+1 in column c (lower index in the low half), hi at t_hi, lo at
// t_hi + CHI/2.
template <int CHI, bool F16>
__device__ __forceinline__ void write_A_tmem(uint32_t t_hi, const float (&v)[CHI]) {
#pragma unroll
    for (int c0 = 0; c0 < CHI; c0 += 64) {
        uint32_t h[32], l[32];
#pragma unroll
        for (int p = 0; p < 32; ++p) split2<F16>(v[c0 + 2 * p], v[c0 + 2 * p + 1], h[p], l[p]);
        tmem_st_2x32(t_hi + (uint32_t)(c0 / 2), t_hi + (uint32_t)(CHI / 2 + c0 / 2), h, l);
    }
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
template <int CHI, int MODE, bool F16>
__global__ void __launch_bounds__(NT, 1)
    k_tc(const __grid_constant__ CUtensorMap map, const Args a) {
    using C = Cfg<CHI, F16>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t stage0 = sa(base);
    uint64_t *bars = (uint64_t *)(base + NS * C::STAGE);
    const uint32_t bar0 = sa(bars);
    // bars: full[0..NS), empty[0..NS), mma_done
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (NS + s); };
    const uint32_t done_bar = bar0 + 8u * (2 * NS);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NS + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    uint32_t *bits = (uint32_t *)(base + NS * C::STAGE + C::CTRL);
    // site table: low 16 bits spin q[k mod N], high 16 bits the prescale c_k
    uint32_t *tab = bits + 4 * a.N;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t c_raw = (int64_t)blockIdx.x * NT + tid;
    const bool active = c_raw < a.B;
    const int64_t c = active ? c_raw : a.B - 1;
    const int j = (MODE == M_ROWS) ? (int)blockIdx.y : 0;
    const int N = a.N;
    const int span = (a.R - 1) * N + 1;
    const int rbase = a.kmin;  // first site the right stack holds
    const long long total_steps = n_steps_of<MODE>(a, j);
    const long long total_atoms = total_steps * C::KA;

    if (warp == 0) tmem_alloc(sa(tmem_slot), C::TALLOC);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    for (int k = tid; k < a.L; k += NT)
        tab[k] = ((uint32_t)__ldg(a.path ? a.path + k : a.q + (k % N)) & 0xffffu) |
                 ((uint32_t)(__ldg(a.cexp + k) & 0xffff) << 16);
    // spin bits: word (i, warp) holds bit (row & 31) = s_i of that row's chain
    for (int i = 0; i < N; ++i) {
        const uint32_t w = __ballot_sync(FULL, a.spins_in[c * N + i] != 0);
        if (lane == 0) bits[i * 4 + warp] = w;
    }
    auto spin = [&](int i) -> int { return (int)((bits[i * 4 + warp] >> lane) & 1u); };
    auto site_spin = [&](int k) -> int { return (int)(tab[k] & 0xffffu); };
    auto site_cexp = [&](int k) -> int { return (int)(int16_t)(tab[k] >> 16); };

    // start vector
    float v[CHI];
    int64_t E = 0;      // exponent of the current row
    int64_t El = 0;     // sweep: exponent of l_{jj-1}
    int64_t Ekeep = 0, Eflip = 0;
    double pm = 0.0;
    int64_t pe = 0, acc_count = 0;
    if (MODE == M_ROWS) {
        if (j == 0) {
            load_vec<CHI>(a.bl, v);
        } else {
            const size_t jm = (size_t)(j > 0 ? j - 1 : 0);
            load_vec<CHI>(a.lstack + ((size_t)c * N + jm) * CHI, v);
            E = a.lexp[(size_t)c * N + jm];
        }
    } else if (MODE == M_RIGHT || MODE == M_SWEEP) {
        load_vec<CHI>(a.br, v);
        if (active) {
            store_vec<CHI>(a.rstack + ((size_t)c * a.nr + (a.nr - 1)) * CHI, v);
            a.rexp[(size_t)c * a.nr + (a.nr - 1)] = 0;
        }
        if (MODE == M_SWEEP) {
            pm = a.state[c].mant;
            pe = a.state[c].exp2;
            if (N == 1) load_vec<CHI>(a.bl, v);  // no right-environment steps
        }
    } else {
        load_vec<CHI>(a.bl, v);
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes
    const uint32_t ta = tw + (uint32_t)C::A_COL;                // this warp's rows of A
    if (total_steps > 0) write_A_tmem<CHI, F16>(ta, v);
    tc_before();
    __syncthreads();
    tc_after();

    // producer (thread 0): cursor over atoms; atom g = step * KA + at
    long long g_issued = 0, g_waited = 0;
    Cursor pc = cursor_start<MODE>(a, j);
    int p_at = 0;
    auto issue_next = [&]() {
        const long long g = g_issued;
        const int st = (int)(g % NS);
        const int y_hi = ((pc.form * 2 + 0) * a.L + pc.k) * 2 * CHI;
        const int y_lo = ((pc.form * 2 + 1) * a.L + pc.k) * 2 * CHI;
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
    if (tid == 0) {
        while (g_issued < total_atoms && g_issued < NS) issue_next();
    }

    Cursor cc = cursor_start<MODE>(a, j);
    bool aborted = false;

    for (long long t = 0; t < total_steps; ++t) {
        // ---------------- MMA issue (thread 0)
        if (tid == 0) {
            for (int at = 0; at < C::KA; ++at) {
                const long long g = t * C::KA + at;
                const int st = (int)(g % NS);
                if (!mbar_wait(full_bar(st), (uint32_t)((g / NS) & 1), a.wait_limit)) {
                    atomicOr(a.err, 1);
                    *abort_flag = 1;
                    break;
                }
                g_waited = g + 1;
                tc_after();
                const uint32_t b_hi = stage0 + (uint32_t)st * C::STAGE, b_lo = b_hi + C::BOX;
                const uint32_t a_hi = tmem + (uint32_t)C::A_COL, a_lo = a_hi + (uint32_t)(CHI / 2);
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                    const uint32_t ao = (uint32_t)(at * 32 + kb * 8);
                    const uint32_t bo = (uint32_t)(kb * 32);
                    mma_f16_ts(tmem, a_hi + ao, sdesc(b_hi + bo), C::IDESC, (at | kb) != 0 ? 1u : 0u);
                    mma_f16_ts(tmem, a_hi + ao, sdesc(b_lo + bo), C::IDESC, 1u);
                    mma_f16_ts(tmem, a_lo + ao, sdesc(b_hi + bo), C::IDESC, 1u);
                }
                mma_commit(empty_bar(st));
            }
            mma_commit(done_bar);
            // refill: each stage as soon as the MMAs that read it are done
            if (!*abort_flag) {
                for (int at = 0; at < C::KA; ++at) {
                    const long long g = t * C::KA + at;
                    if (g + NS >= total_atoms) break;
                    const int st = (int)(g % NS);
                    if (!mbar_wait(empty_bar(st), (uint32_t)((g / NS) & 1), a.wait_limit)) {
                        atomicOr(a.err, 1);
                        *abort_flag = 1;
                        break;
                    }
                    issue_next();
                }
            }
        }
        // ---------------- wait for the accumulator
        if (!mbar_wait(done_bar, (uint32_t)(t & 1), a.wait_limit)) {
            atomicOr(a.err, 1);
            *abort_flag = 1;
        }
        tc_after();
        __syncwarp();
        bool write_next = false;
        const int k = cc.k;
        const int sk = site_spin(k);
        const int ck = site_cexp(k);
        // ---------------- epilogue
        if (MODE == M_ROWS) {
            const int iflip = (j < N) ? site_spin(j) : -1;
            acc_select<CHI>(tw, spin(sk) ^ (sk == iflip ? 1 : 0), v);
            E += renorm<CHI>(v) - ck;
            write_next = (t + 1 < total_steps);
        } else if (MODE == M_LEFT) {
            acc_select<CHI>(tw, spin(sk), v);
            E += renorm<CHI>(v) - ck;
            if (active) {
                store_vec<CHI>(a.lstack + ((size_t)c * N + k) * CHI, v);
                a.lexp[(size_t)c * N + k] = (int32_t)E;
            }
            write_next = (t + 1 < total_steps);
        } else if (MODE == M_RIGHT) {
            acc_select<CHI>(tw, spin(sk), v);
            E += renorm<CHI>(v) - ck;
            if (active) {
                store_vec<CHI>(a.rstack + ((size_t)c * a.nr + (k - rbase)) * CHI, v);
                a.rexp[(size_t)c * a.nr + (k - rbase)] = (int32_t)E;
            }
            write_next = (t + 1 < total_steps);
        } else if (MODE == M_INIT) {
            acc_select<CHI>(tw, spin(sk), v);
            E += renorm<CHI>(v) - ck;
            write_next = (t + 1 < total_steps);
        } else {  // M_SWEEP
            if (cc.form == 1) {  // right environment of the last block
                acc_select<CHI>(tw, spin(sk), v);
                E += renorm<CHI>(v) - ck;
                if (active) {
                    store_vec<CHI>(a.rstack + ((size_t)c * a.nr + (k - rbase)) * CHI, v);
                    a.rexp[(size_t)c * a.nr + (k - rbase)] = (int32_t)E;
                }
                if (cc.tt == N - 2) {  // next: proposal 0 starts from b_L
                    load_vec<CHI>(a.bl, v);
                    El = 0;
                }
                write_next = true;
            } else {
                const int jj = cc.jj;
                const int iq = site_spin(jj);
                if (cc.i == 0) {
                    const int si = spin(iq);
                    // unflipped continuation: l_jj if the proposal is rejected
                    acc_select<CHI>(tw, si, v);
                    Ekeep = El + renorm<CHI>(v) - ck;
                    if (active) {
                        store_vec<CHI>(a.lstack + ((size_t)c * N + jj) * CHI, v);
                        a.lexp[(size_t)c * N + jj] = (int32_t)Ekeep;
                    }
                    // flipped start of the proposal row
                    acc_select<CHI>(tw, si ^ 1, v);
                    Eflip = El + renorm<CHI>(v) - ck;
                    if (active) {
                        store_vec<CHI>(a.tmp + (size_t)c * CHI, v);
                        a.tmp_exp[c] = (int32_t)Eflip;
                    }
                    E = Eflip;
                } else {
                    acc_select<CHI>(tw, spin(sk) ^ (sk == iq ? 1 : 0), v);
                    E += renorm<CHI>(v) - ck;
                }
                if (cc.i + 1 < span) {
                    write_next = true;
                } else {
                    // Metropolis decision of proposal jj (spin iq)
                    const float *r = a.rstack + ((size_t)c * a.nr + jj) * CHI;
                    int64_t Ep = E + a.rexp[(size_t)c * a.nr + jj];
                    double m = dot<CHI>(v, r);
                    normalize_scalar(m, Ep);
                    const double ratio = ldexp(m / pm, (int)(Ep - pe));
                    const double x = rttd::mcmc_uniform(a.seed, (uint64_t)(a.chain0 + c),
                                                        (uint64_t)(a.sweep0 + cc.sw), (uint64_t)jj);
                    const bool accept = active && (x < ratio * ratio);
                    if (accept) {
                        pm = m;
                        pe = Ep;
                        ++acc_count;
                        load_vec<CHI>(a.tmp + (size_t)c * CHI, v);
                        store_vec<CHI>(a.lstack + ((size_t)c * N + jj) * CHI, v);
                        a.lexp[(size_t)c * N + jj] = (int32_t)Eflip;
                        El = Eflip;
                    } else {
                        El = Ekeep;
                    }
                    const uint32_t flips = __ballot_sync(FULL, accept);
                    if (lane == 0) bits[iq * 4 + warp] ^= flips;
                    __syncwarp();
                    if (jj + 1 < N) {  // next proposal starts from l_jj
                        load_vec<CHI>(a.lstack + ((size_t)c * N + jj) * CHI, v);
                        write_next = true;
                    } else if (cc.sw + 1 < a.n_sweeps) {  // next sweep
                        load_vec<CHI>(N > 1 ? a.br : a.bl, v);
                        E = 0;
                        El = 0;
                        write_next = true;
                    }
                }
            }
        }
        if (write_next) write_A_tmem<CHI, F16>(ta, v);
        cursor_next<MODE>(cc, a, span);
        tc_before();
        __syncthreads();
        tc_after();
        if (*abort_flag) {
            aborted = true;
            break;
        }
    }

    // ---------------- final contraction / outputs
    if (!aborted) {
        if (MODE == M_ROWS) {
            const int rq = row_end(a, j) + 1 - a.kmin;  // r_{end+1}; b_R for j = N
            int64_t Ep = E + a.rexp[(size_t)c * a.nr + rq];
            double m = dot<CHI>(v, a.rstack + ((size_t)c * a.nr + rq) * CHI);
            normalize_scalar(m, Ep);
            if (active) {
                a.rows_mant[c * (N + 1) + j] = m;
                a.rows_exp[c * (N + 1) + j] = Ep;
            }
        } else if (MODE == M_INIT) {
            double m = dot<CHI>(v, a.br);
            int64_t Ep = E;
            normalize_scalar(m, Ep);
            if (active) {
                if (a.state) {
                    a.state[c].mant = m;
                    a.state[c].exp2 = Ep;
                }
                if (a.log_abs)
                    a.log_abs[c] = (m == 0.0) ? -INFINITY : (double)Ep * 0.6931471805599453 + log(fabs(m));
                if (a.sign) a.sign[c] = (m > 0.0) ? 1 : ((m < 0.0) ? -1 : 0);
            }
        } else if (MODE == M_SWEEP) {
            if (active) {
                for (int i = 0; i < N; ++i) a.spins_out[c * N + i] = (uint8_t)spin(i);
                a.state[c].mant = pm;
                a.state[c].exp2 = pe;
                if (a.n_accept) a.n_accept[c] += acc_count;
            }
        }
    }
    // ---------------- teardown: drain own copies (bounded), free TMEM
    if (tid == 0 && aborted) {
        for (long long g = g_waited; g < g_issued; ++g)
            mbar_wait(full_bar((int)(g % NS)), (uint32_t)((g / NS) & 1), a.wait_limit);
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tmem_dealloc(tmem, C::TALLOC);
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

__device__ __forceinline__ void named_sync_256() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
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
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
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
    const size_t smem = tcd::Cfg<CHI, F16>::smem_bytes(a.N, a.L);
    cudaError_t e = cudaFuncSetAttribute(tcd::k_tc<CHI, MODE, F16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tcd::k_tc<CHI, MODE, F16><<<grid, tcd::NT, smem, st>>>(p->map, a);
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
    cudaError_t e;
    if ((e = cudaMalloc((void **)&p->d_B, Bh.size() * sizeof(uint16_t))) != cudaSuccess)
        return status_of(e, "tc plan: tensors");
    if ((e = cudaMemcpy(p->d_B, Bh.data(), Bh.size() * sizeof(uint16_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return status_of(e, "tc plan: tensors copy");
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
    const cuuint64_t gdim[2] = {(cuuint64_t)chi, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)chi * sizeof(uint16_t)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)(2 * chi)};
    const cuuint32_t estride[2] = {1u, 1u};
    CUresult r = enc(&p->map,
                     p->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     p->d_B, gdim, gstride, box, estride,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        rtt_set_error("cuTensorMapEncodeTiled failed");
        return RTT_ERR_CUDA;
    }
    return RTT_OK;
}

void tc_plan_destroy(rtt_s *h) {
    TcPlan *p = h->tc;
    if (!p) return;
    cudaFree(p->d_B);
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
    cudaError_t e = launch_chi<tcd::M_ROWS>(h->tc, a, dim3(tiles(B), h->N + 1), st);
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
    if (!h->periodic && !(p->chi == 64 && h->R >= 2 && h->N >= 2)) {
        prof_end(h, KID_TC_SWEEP, st);
        rtt_set_error("rtt_mcmc_sweep: tensor-core sweeps on a general path need chi = 64 and "
                      "at least two replicas");
        return RTT_ERR_UNSUPPORTED;
    }
    if (p->chi == 64 && h->R >= 2 && h->N >= 2) {
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
