// Triplet and quadruplet contractions on the 5th-generation tensor cores
// (tcgen05, sm_103a).
//
// The real-space sums of Eq. Jeong_BI, num[a,b,c] = sum_x I_a I_b I_c, are a
// matrix product D[(b,c)][n] = sum_x P_bc(x) R_n(x) with the outer pair
// products P_bc = I_b I_c formed on the fly (M = 128 outer pairs per tile),
// inner rows R_n that are single bins (bispectrum) or pair products I_a I_b
// (trispectrum, Eq. Jeong_gen with p = 4) on N, and K = points x.  Per
// pipeline step of 64 or 128 points:
//   * one loader thread streams every bin's shell field of the step into a
//     ring of shared-memory stages with 2-D TMA loads (128-byte swizzle);
//   * producer warps split the inner rows into BF16 hi/lo (operand B, 128-byte
//     swizzled K-major tiles in shared memory) and form the outer pair products
//     of their tensor-memory lane, split them into BF16 hi/lo and store them
//     into tensor memory (operand A) with tcgen05.st;
//   * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) for
//     hi*hi + hi*lo + lo*hi (BF16x3; hi*hi alone for plain BF16) into FP32
//     accumulators in tensor memory, one 128 x Npad block per pair tile; the
//     hi and lo rows of B sit side by side in each K-atom, so where the
//     doubled accumulators fit, A_hi x [B_hi; B_lo] (N = 2 Npad) and A_lo x
//     B_hi take two MMAs per K step instead of three, and a single tile of
//     at most 64 pairs stacks A's hi and lo rows on M for one MMA per K step
//     (which also forms lo*lo);
//   * every 1,024 points the producers read the accumulators back
//     (tcgen05.ld) into compensated (Kahan) FP32 sums per item in shared
//     memory, after the next step's operands are handed off.
// An MMA of M = 128 and K = 16 occupies the issuing thread for about 100
// cycles whatever N is up to 160 (measured), so the fewer and wider the MMAs
// the better; the producers run up to three steps ahead of them (operand-B
// ring of up to 4 stages).  In a single-tile trispectrum pass the inner pair
// rows that are outer rows too are stored into operand B by the operand-A
// warps that form the same products.
// Each CTA owns a contiguous range of points; its sums go to its own row of
// the FP64 partial buffer, reduced across CTAs in a fixed order.  Which of a
// triplet's (or quadruplet's) pairs forms the outer row is chosen by a greedy
// set cover (pair_cover.cpp) to keep the 128-row tiles few.
//
// Every wait on an mbarrier is bounded (about one second of clock cycles by
// default, FBS_OPT_TC_WAIT_LIMIT for the hand-offs between roles); on
// timeout the CTA records an error code, stops issuing loads and MMAs, waits
// (bounded) for those in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <array>
#include <iterator>
#include <map>
#include <set>
#include <utility>

#include "fbs_internal.h"
#include "pair_cover.h"

namespace fbs {

namespace {

constexpr int KC = 64;              // points per chunk (one 128-byte swizzle row of BF16)
constexpr int kStageLd = KC + 4;    // staged row stride in floats (bank spread)
constexpr long long kWaitCycles = 2000000000LL;

constexpr int kMaxInner = 256;       // operand-B rows (N of the MMA) at most

// One outer pair (rows of operand A) and the inner rows it closes with.
struct TcPair {
    int b, c, first, pad;
    unsigned mask[kMaxInner / 32];  // bit n: inner row n closes a polygon with (b, c)
};

// One contraction: outer pairs x inner rows.  Inner row n is the single bin
// in0[n] (in1[n] < 0, bispectrum) or the pair product in0[n] x in1[n]
// (trispectrum).
struct TcJob {
    TcPair *d_pairs = nullptr;
    int2 *d_inner = nullptr;
    int *d_iout = nullptr;   // job item (pair-major, inner rows ascending) -> output column
    int npairs = 0, ntiles = 0, ninner = 0, Npad = 0, maxloc = 0, maxtiles = 0;
    std::vector<int> grp;  // tile ranges of the CTA groups
    int *d_grp = nullptr;
    bool built = false, usable = false;
    int variant = 0;       // pair assignment the tables were built with (FBS_OPT_TC_PAIRS)
    int *d_ifeed = nullptr;  // single-tile jobs: per outer row, the inner pair row of the same product, or -1
    int nsingle = 0;         // inner rows built from the field stage with d_ifeed (a prefix of the inner rows)
    int last_merged = -1, last_ka = 0;  // MMA shape of the latest launch (diagnostics)
    int last_bfa = 0;                   // inner pair rows the latest launch took from operand A
    int last_nsb = 0, last_nstg = 0, last_nst = 0;  // its B, field and A stage counts
};

struct WideRight {
    int x, y, first, pad;    // product I_x I_y; index of its first item
    unsigned long long mask; // bit l: left row l forms an item with this right row
};

struct WideJob {
    int nleft = 0, nright = 0, nitems = 0, maxloc = 0;
    int2 *d_left = nullptr;
    WideRight *d_rights = nullptr;
    int *d_item_out = nullptr;
    bool built = false, usable = false;
};

struct TcState {
    TcJob trip, quad, fused;
    WideJob wtrip, wquad;
    int *d_err = nullptr;     // the root plan's flags: [0] this evaluation's wait-timeout code, [1] sticky copy
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major, 128-byte swizzled operand tile: rows of 128 B (64 BF16 along K),
// 8-row groups 1024 B apart.  Start address must sit in a 1024-B aligned tile
// (plus the 32-B K-step offset).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;   // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *gptr, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gptr), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Byte offset of (row, 16-byte chunk j) in a 128-byte swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_off(int row, int j) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((j ^ (row & 7)) << 4));
}

// Split two FP32 values into BF16 hi (round to nearest) and lo = bf16(v - hi)
// with packed FP32x2 arithmetic: v - hi is exact in FP32 (hi is v rounded to
// 8 significant bits), so one fused multiply-add by -1 gives it; the packed
// and the scalar forms round identically.
__device__ __forceinline__ void split2(float2 v, uint32_t &h, uint32_t &l) {
    const __nv_bfloat162 hb = __float22bfloat162_rn(v);
    h = *reinterpret_cast<const uint32_t *>(&hb);
    const float2 hf = make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xffff0000u));
    const __nv_bfloat162 lb = __float22bfloat162_rn(__ffma2_rn(hf, make_float2(-1.f, -1.f), v));
    l = *reinterpret_cast<const uint32_t *>(&lb);
}

// Products a*b of 8 values (two float4 pairs) split into BF16 hi/lo words.
__device__ __forceinline__ void mul_split8(float4 a0, float4 a1, float4 b0, float4 b1, uint32_t *h, uint32_t *l) {
    split2(__fmul2_rn(make_float2(a0.x, a0.y), make_float2(b0.x, b0.y)), h[0], l[0]);
    split2(__fmul2_rn(make_float2(a0.z, a0.w), make_float2(b0.z, b0.w)), h[1], l[1]);
    split2(__fmul2_rn(make_float2(a1.x, a1.y), make_float2(b1.x, b1.y)), h[2], l[2]);
    split2(__fmul2_rn(make_float2(a1.z, a1.w), make_float2(b1.z, b1.w)), h[3], l[3]);
}

// Split 8 FP32 values into BF16 hi (round to nearest) and lo = bf16(v - hi).
__device__ __forceinline__ void split8(const float *v, uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        float2 hf = __bfloat1622float2(hb);
        __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
        h[i] = *reinterpret_cast<uint32_t *>(&hb);
        l[i] = *reinterpret_cast<uint32_t *>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

}  // namespace

// Warp roles of the narrow kernel: warps 0..15 produce (operand B into
// shared memory, the pair products into tensor memory, the accumulator
// flushes); warp 16 allocates tensor memory and one of its threads issues
// every MMA; one thread of warp 17 streams the shell fields of each chunk
// into a ring of shared-memory stages with TMA.  Every hand-off is an
// mbarrier; no role waits on a CTA-wide barrier inside the main loop.
constexpr int kProdWarps = 16;            // A-operand warps (AW) + operand-B warps (16 - AW)
constexpr int kMmaWarp = kProdWarps;
constexpr int kLoadWarp = kProdWarps + 1;
constexpr int kTcThreads = (kProdWarps + 2) * 32;
constexpr int kAStageCols = 64;           // per K-atom: 32 columns hi + 32 columns lo (64 BF16 per row each)
constexpr int kMaxAStages = 3;
constexpr int kMaxFieldStages = 4;
constexpr int kMaxBStages = 4;

struct TcBars {
    uint64_t sfull[kMaxFieldStages], sempty[kMaxFieldStages];
    uint64_t full[kMaxAStages], empty[kMaxAStages], bfull[kMaxBStages], bempty[kMaxBStages], accr, accf;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 2-D tiled TMA load (x = point, y = bin) into shared memory; completion is
// counted in bytes on the mbarrier.  Points past the tensor's end read zero.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait that gives up at once after any other wait of the CTA timed
// out (the abort flag is sticky), so no role can strand another.
// `limit` is the launch's hand-off wait limit in clock cycles (about one
// second by default; a plan option shortens it to exercise this path).
__device__ __forceinline__ bool role_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *err, int code, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;  // ready: no clock read, no flag read
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            atomicExch(err, code);
            return false;
        }
    }
    return true;
}

// Position in a ring of S slots: the slot and the parity of its use count
// (the phase a consumer waits for; a producer refilling the slot waits for
// the opposite parity once every slot has been used).
template <int S>
struct Ring {
    int slot = 0;
    uint32_t phase = 0;
    bool warm = false;
    __device__ __forceinline__ void next() {
        if (++slot == S) {
            slot = 0;
            phase ^= 1u;
            warm = true;
        }
    }
};

// The same for a ring whose size is a launch parameter.
struct RingN {
    int slot = 0, n;
    uint32_t phase = 0;
    bool warm = false;
    __device__ explicit RingN(int size) : n(size) {}
    __device__ __forceinline__ void next() {
        if (++slot == n) {
            slot = 0;
            phase ^= 1u;
            warm = true;
        }
    }
};

__device__ __forceinline__ void tmem_st8a(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
        "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
        : "memory");
}

// MMA with a compile-time accumulate flag (no predicate setup in the issue loop).
template <bool ACC>
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc) {
    if (ACC)
        asm volatile(
            "{\n .reg .pred p;\n setp.eq.u32 p, 1, 1;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b), "r"(idesc)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.eq.u32 p, 1, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b), "r"(idesc)
            : "memory");
}

// Compensated (Kahan) FP32 running sum: x = sum, y = compensation; the
// value is x - y.  Explicit round-to-nearest operations keep the compiler
// from contracting or reassociating them.
__device__ __forceinline__ void kahan_add(float2 &a, float v) {
    const float y = __fsub_rn(v, a.y);
    const float t = __fadd_rn(a.x, y);
    a.y = __fsub_rn(__fsub_rn(t, a.x), y);
    a.x = t;
}

// A field stage holds 64 KA points of every bin as 2 KA boxes of 32 points,
// each [rows][128 B] in the TMA 128-byte swizzle: 16-byte chunk J (points
// 4J..4J+3) of bin row b at chunk (J mod 8) ^ (b mod 8) of the row in box J / 8.

// The values of one operand-B unit (inner row with bins `in`, 8-point group
// of the step whose 16-byte chunks 2j, 2j + 1 sit in the 32-point box at
// `box`, chunk 2j at position jp before the swizzle): the x bin's 8 values
// and, for a pair row, the y bin's.  Chunk 2j + 1 of a row is chunk 2j with
// bit 4 of the offset flipped (jp is even).
struct BUnit {
    float4 x0, x1, y0, y1;
};

__device__ __forceinline__ void b_unit_load(const unsigned char *box, int jp, int2 in, BUnit &u) {
    const uint32_t ox = (uint32_t)in.x * 128u + ((uint32_t)(jp ^ (in.x & 7)) << 4);
    u.x0 = *reinterpret_cast<const float4 *>(box + ox);
    u.x1 = *reinterpret_cast<const float4 *>(box + (ox ^ 16u));
    if (in.y >= 0) {
        const uint32_t oy = (uint32_t)in.y * 128u + ((uint32_t)(jp ^ (in.y & 7)) << 4);
        u.y0 = *reinterpret_cast<const float4 *>(box + oy);
        u.y1 = *reinterpret_cast<const float4 *>(box + (oy ^ 16u));
    }
}

// The unit's values (a single bin, or the product of two bins) split into
// BF16 hi/lo and stored at byte offset `off` of the hi and lo tiles.
__device__ __forceinline__ void b_unit_store(const BUnit &u, bool pair, unsigned char *bh, unsigned char *bl,
                                             uint32_t off) {
    uint32_t h[4], l[4];
    if (pair) {
        mul_split8(u.x0, u.x1, u.y0, u.y1, h, l);
    } else {
        split2(make_float2(u.x0.x, u.x0.y), h[0], l[0]);
        split2(make_float2(u.x0.z, u.x0.w), h[1], l[1]);
        split2(make_float2(u.x1.x, u.x1.y), h[2], l[2]);
        split2(make_float2(u.x1.z, u.x1.w), h[3], l[3]);
    }
    *reinterpret_cast<uint4 *>(bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(bl + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Operand B of one pipeline step by W warps (wb = 0..W-1 among them): the
// C = 8 KA eight-point groups go to the warps (W / C warps per group), inner
// rows 0..nrows-1 to their lanes.  Each unit is split into BF16 hi/lo in the
// 128-byte-swizzled K-major tile of K-atom j / 8.
template <int W, int KA>
__device__ __forceinline__ void build_b(const unsigned char *st, int half_bytes, const int2 *s_inner, int nrows,
                                        int wb, int lane, unsigned char *bh, unsigned char *bl, int atom_stride) {
    constexpr int C = 8 * KA;
    static_assert(W % C == 0, "operand-B warps must cover the eight-point groups evenly");
    const int j = wb % C;
    const unsigned char *box = st + ((2 * j) >> 3) * half_bytes;
    const int jp = (2 * j) & 7;
    const uint32_t dj = (uint32_t)((j >> 3) * atom_stride);
    for (int row = lane + 32 * (wb / C); row < nrows; row += 32 * (W / C)) {
        const int2 in = s_inner[row];
        BUnit u;
        b_unit_load(box, jp, in, u);
        b_unit_store(u, in.y >= 0, bh, bl, dj + sw128_off(row, j & 7));
    }
}

// grid: (G point-range CTAs, groups of pair tiles).  One CTA per SM.
// NST: A stages in tensor memory; NSTG: field stages in shared memory;
// nsb (launch parameter, 2..4): operand-B stages in shared memory.
// stacked (one pair tile of at most 64 pairs, BF16x3, merged B): operand A
// holds hi of pair r in row r and lo of pair r in row r + 64 (the warps of
// lane quarters 2 and 3 form the same products), so one MMA per K step with
// N = 2 Npad gives hi*hi, hi*lo (rows 0..63) and lo*hi, lo*lo (rows
// 64..127); rows r + 64 are summed into a second set of compensated sums.
// ifeed (null, or with a single pair tile and AW = 16): per outer row, the
// inner pair row with the same product (-1: none); the operand-A thread of
// that row also stores its hi/lo values into operand B, and the operand-B
// build covers inner rows 0..nbuild-1 only.
// AW: warps forming the pair products of operand A (4 per TMEM lane quarter
// x 16 points, or 2 x 32 points); with AW = 16 they also build operand B,
// with AW = 8 the other 8 producer warps build operand B concurrently.
// KA: 64-point K-atoms per chunk (1 or 2): a chunk is 64 KA points, staged as
// 2 KA TMA boxes of 32 points, with one swizzled B tile per atom and A stages
// of 64 KA tensor-memory columns.
template <int NST, int NSTG, int AW, int KA, bool FEED>
__global__ void __launch_bounds__(kTcThreads, 1)
    contract_tc_kernel(const __grid_constant__ CUtensorMap fmap, long long npts, int nbins, int Npad,
                       int tstride, int ninner, const int2 *__restrict__ inner,
                       const TcPair *__restrict__ pairs, int npairs,
                       const int *__restrict__ grp_tile0, const int *__restrict__ iout,
                       int nitems_total, double *__restrict__ part, int x3, int flush_every,
                       int *__restrict__ err, long long wait_limit, int part_rows, int merged, int nsb,
                       const int *__restrict__ ifeed, int nbuild, int stacked_arg) {
    static_assert(AW == 16 || AW == 8, "A-operand warps: 16 or 8");
    static_assert(!FEED || AW == 16, "inner pair rows from operand A: the A warps build operand B");
    static_assert(KA == 1 || KA == 2, "K-atoms per chunk: 1 or 2");
    constexpr int BW = kProdWarps - AW;   // operand-B warps (0: the A warps build it)
    const int stacked = FEED ? 0 : stacked_arg;  // the host never stacks with the feed
    constexpr int KCH = KC * KA;          // points per chunk
    constexpr int PPT = 4 * KCH / AW;     // points of a row per A thread per tile
    constexpr int ACOLS = kAStageCols * KA;  // tensor-memory columns of one A stage
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ TcBars bars;
    __shared__ int2 s_inner[kMaxInner];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = blockIdx.y;
    const int t0 = grp_tile0[g], t1 = grp_tile0[g + 1];
    const int ntl = t1 - t0;
    const int p_first = t0 * 128;
    const int p_last = min(npairs, t1 * 128);
    const int it0 = pairs[p_first].first;
    int nloc = 0;
    if (p_last > p_first) {
        nloc = pairs[p_last - 1].first - it0;
#pragma unroll
        for (int w = 0; w < kMaxInner / 32; ++w) nloc += __popc(pairs[p_last - 1].mask[w]);
    }

    // ---- shared memory: B tiles and field stages (1024-aligned), sums, pair bins
    uintptr_t base = (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023;
    unsigned char *sm = reinterpret_cast<unsigned char *>(base);
    const int b_tile = Npad * 128;      // one K-atom of operand B (hi or lo)
    // one B stage holds, per K-atom, the hi rows then the lo rows (one tile of
    // 2 Npad rows: a single MMA with N = 2 Npad multiplies both halves)
    const int b_stage = KA * b_tile;    // hi (or lo) part of one B stage
    const int b_atom2 = 2 * b_tile;     // one K-atom: hi tile, then lo tile
    unsigned char *const Bh0 = sm;      // stage sb (< nsb) at Bh0 + 2 sb b_stage
    const int half_bytes = ((nbins + 7) & ~7) * 128;  // one 32-point TMA box of all bins
    const int stage_bytes = 2 * KA * half_bytes;
    unsigned char *const stg = sm + 2 * nsb * b_stage;
    float2 *acc = reinterpret_cast<float2 *>(stg + NSTG * stage_bytes);
    float2 *acc2 = acc + nloc;  // stacked: the sums of rows 64..127 (lo * B)
    int2 *pbc = reinterpret_cast<int2 *>(acc + (stacked ? 2 : 1) * nloc);  // (b, c) of every row of every tile

    const int acc_cols = ((ntl * tstride + 31) / 32) * 32;
    const int tmem_cols_needed = acc_cols + NST * ACOLS;
    int ncols = 32;
    while (ncols < tmem_cols_needed) ncols <<= 1;

    if (tid == 0) {
        for (int i = 0; i < NSTG; ++i) {
            mbar_init(&bars.sfull[i], 1);
            mbar_init(&bars.sempty[i], kProdWarps);
        }
        for (int i = 0; i < NST; ++i) {
            mbar_init(&bars.full[i], AW);
            mbar_init(&bars.empty[i], 1);
        }
        for (int i = 0; i < nsb; ++i) {
            mbar_init(&bars.bfull[i], BW > 0 ? BW : AW);
            mbar_init(&bars.bempty[i], 1);
        }
        mbar_init(&bars.accr, 1);
        mbar_init(&bars.accf, AW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < (stacked ? 2 : 1) * nloc; i += kTcThreads) acc[i] = make_float2(0.f, 0.f);
    for (int i = tid; i < ninner; i += kTcThreads) s_inner[i] = inner[i];
    for (int i = tid; i < ntl * 128; i += kTcThreads) {
        const int p = p_first + i;
        pbc[i] = p < npairs ? make_int2(pairs[p].b, pairs[p].c) : make_int2(-1, -1);
    }
    for (int i = tid; i < 2 * nsb * b_stage / 16; i += kTcThreads) {  // padding rows of B stay zero
        int o = i % (b_tile / 16);
        if ((o * 16) / 128 >= ninner) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abortp = &abort_flag;

    const long long nchunks = (npts + KCH - 1) / KCH;
    constexpr bool bfa = FEED;  // the host launches FEED with ifeed and one pair tile only
    const long long c0 = nchunks * blockIdx.x / gridDim.x;
    const long long c1 = nchunks * (blockIdx.x + 1) / gridDim.x;

    if (warp == kLoadWarp) {
        // ================= field loader (one thread) =================
        if (lane == 0 && c0 < c1) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&fmap)) : "memory");
            const uint32_t bytes = 2u * KA * (uint32_t)nbins * 128u;
            Ring<NSTG> rs;
            long long issued = 0;
            for (long long ci = c0; ci < c1; ++ci) {
                if (rs.warm && !role_wait(&bars.sempty[rs.slot], rs.phase ^ 1u, abortp, err, 10, wait_limit)) break;
                // After an abort a producer warp may hand a stage back before its load
                // landed (it set the flag before arriving, so the flag is visible
                // here): never issue a second load into a slot, so every slot has
                // at most one copy in flight and the drain below covers all of them.
                if (*abortp) break;
                const uint32_t dst = smem_u32(stg + rs.slot * stage_bytes);
                const int x = (int)(ci * KCH);
                mbar_expect_tx(&bars.sfull[rs.slot], bytes);
#pragma unroll
                // field blockIdx.z of a batch: its bins are rows nbins * blockIdx.z of the map
                for (int h = 0; h < 2 * KA; ++h)
                    tma_load_2d(dst + h * half_bytes, &fmap, x + 32 * h, (int)blockIdx.z * nbins,
                                &bars.sfull[rs.slot]);
                rs.next();
                ++issued;
            }
            // every copy into this CTA's shared memory has landed before it exits (own limit)
            for (long long j = issued > NSTG ? issued - NSTG : 0; j < issued; ++j) {
                const int slot = (int)(j % NSTG);
                if (!mbar_wait(&bars.sfull[slot], (uint32_t)((j / NSTG) & 1))) atomicExch(err, 16);
            }
        }
    } else if (warp == kMmaWarp) {
        // ================= MMA issuer (one thread) =================
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, Npad);
            const uint32_t idesc2 = idesc_bf16(128, 2 * Npad);  // hi and lo rows of B together
            Ring<NST> ra;
            RingN rb(nsb);
            long long nfl = 0;
            int last_slot = -1;
            uint32_t last_phase = 0;
            bool fresh = true;
            int since = 0;
            for (long long ci = c0; ci < c1; ++ci) {
                const int sb = rb.slot;
                const bool okb = role_wait(&bars.bfull[sb], rb.phase, abortp, err, 11, wait_limit);
                const uint64_t dbh = sdesc_sw128(smem_u32(Bh0 + 2 * sb * b_stage));
                const uint64_t dbl = dbh + (uint64_t)((unsigned)b_tile >> 4);  // the atom's lo rows
                const uint64_t datom = (uint64_t)((unsigned)b_atom2 >> 4);     // next K-atom
                for (int lt = 0; lt < ntl; ++lt) {
                    const int as = ra.slot;
                    const bool oka = role_wait(&bars.full[as], ra.phase, abortp, err, 12, wait_limit);
                    tc_fence_after();
                    if (okb && oka) {  // a failed wait leaves ok false (the abort flag is sticky)
                        const uint32_t d = tmem + (uint32_t)(lt * tstride);
                        const uint32_t ah = tmem + (uint32_t)(acc_cols + as * ACOLS);
                        const uint32_t al = ah + 32u * KA;
                        // k-step k: A columns 8k; B atom k/4 (tile start + 2 b_tile),
                        // start address field + 2 (k mod 4) within the atom (32 bytes).
                        // merged: A_hi x [B_hi; B_lo] (N = 2 Npad) accumulates hi*hi in
                        // columns [0, Npad) and hi*lo in [Npad, 2 Npad); A_lo x B_hi adds
                        // lo*hi to the first half: two MMAs per k-step instead of three.
                        if (stacked) {  // rows 0..63 hi, 64..127 lo of A: one MMA per k-step
                            if (fresh) mma_ts<false>(d, ah, dbh, idesc2);
                            else mma_ts<true>(d, ah, dbh, idesc2);
#pragma unroll
                            for (int k = 1; k < 4 * KA; ++k) {
                                const uint64_t bo = datom * (uint64_t)(k >> 2) + 2u * (k & 3);
                                mma_ts<true>(d, ah + 8u * k, dbh + bo, idesc2);
                            }
                        } else if (merged) {
                            if (fresh) mma_ts<false>(d, ah, dbh, idesc2);
                            else mma_ts<true>(d, ah, dbh, idesc2);
                            mma_ts<true>(d, al, dbh, idesc);
#pragma unroll
                            for (int k = 1; k < 4 * KA; ++k) {
                                const uint64_t bo = datom * (uint64_t)(k >> 2) + 2u * (k & 3);
                                mma_ts<true>(d, ah + 8u * k, dbh + bo, idesc2);
                                mma_ts<true>(d, al + 8u * k, dbh + bo, idesc);
                            }
                        } else {
                            if (fresh) mma_ts<false>(d, ah, dbh, idesc);
                            else mma_ts<true>(d, ah, dbh, idesc);
                            if (x3) {
                                mma_ts<true>(d, ah, dbl, idesc);
                                mma_ts<true>(d, al, dbh, idesc);
                            }
#pragma unroll
                            for (int k = 1; k < 4 * KA; ++k) {
                                const uint64_t bo = datom * (uint64_t)(k >> 2) + 2u * (k & 3);
                                mma_ts<true>(d, ah + 8u * k, dbh + bo, idesc);
                                if (x3) {
                                    mma_ts<true>(d, ah + 8u * k, dbl + bo, idesc);
                                    mma_ts<true>(d, al + 8u * k, dbh + bo, idesc);
                                }
                            }
                        }
                    }
                    mma_commit(&bars.empty[as]);
                    last_slot = as;
                    last_phase = ra.phase;
                    ra.next();
                }
                mma_commit(&bars.bempty[sb]);
                rb.next();
                fresh = false;
                if (++since == flush_every || ci == c1 - 1) {
                    mma_commit(&bars.accr);
                    role_wait(&bars.accf, (uint32_t)(nfl & 1), abortp, err, 13, wait_limit);
                    tc_fence_after();
                    ++nfl;
                    fresh = true;
                    since = 0;
                }
            }
            // drain: every MMA complete before tensor memory is released (own limit)
            if (last_slot >= 0 && !mbar_wait(&bars.empty[last_slot], last_phase)) atomicExch(err, 14);
        }
    } else if (BW > 0 && warp >= AW) {
        // ================= operand-B warps (AW .. 15) =================
        Ring<NSTG> rs;
        RingN rb(nsb);
        for (long long ci = c0; ci < c1; ++ci) {
            role_wait(&bars.sfull[rs.slot], rs.phase, abortp, err, 24, wait_limit);
            const unsigned char *st = stg + rs.slot * stage_bytes;
            const int sb = rb.slot;
            if (rb.warm) role_wait(&bars.bempty[sb], rb.phase ^ 1u, abortp, err, 25, wait_limit);
            // (8 KA when BW = 0 only keeps the never-taken instantiation well formed)
            build_b<(BW > 0 ? BW : 8 * KA), KA>(st, half_bytes, s_inner, ninner, warp - AW, lane,
                                                 Bh0 + 2 * sb * b_stage, Bh0 + 2 * sb * b_stage + b_tile, b_atom2);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.bfull[sb]);
            rb.next();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.sempty[rs.slot]);
            rs.next();
        }
    } else {
        // ================= operand-A warps (0 .. AW-1) =================
        const int q = warp & 3, kq = warp >> 2;  // lane quarter, PPT-point slice of the chunk
        const int r = 32 * q + lane;             // operand-A row (TMEM lane) of this thread
        const int feed = bfa ? ifeed[r] : -1;    // inner row with this row's product (single tile)
        // A warp whose 32 rows are all padding of the only pair tile zeroes its
        // lanes of every A stage once here; nothing rewrites them (the MMAs only
        // read A), so in the loop it takes part in the hand-offs only.
        const bool idle = !stacked && ntl == 1 && 32 * q >= npairs - t0 * 128;
        Ring<NSTG> rs;
        Ring<NST> ra;
        RingN rb(nsb);
        long long nfl = 0;
        int since = 0;
        bool pend = false;  // a flush point has passed; its flush is still due
        auto flush = [&]() {
            role_wait(&bars.accr, (uint32_t)(nfl & 1), abortp, err, 23, wait_limit);
            tc_fence_after();
            if (!*abortp && !idle) {
                float2 *const sums = stacked && r >= 64 ? acc2 : acc;
                for (int lt = 0; lt < ntl; ++lt) {
                    const int p = (t0 + lt) * 128 + (stacked ? (r & 63) : r);
                    const bool valid = p < npairs;
                    const TcPair *pp = pairs + (valid ? p : 0);
                    for (int c8 = 8 * kq; c8 < Npad; c8 += 8 * (AW / 4)) {
                        float v[8];
                        tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(lt * tstride + c8), v);
                        if (merged) {  // hi*lo sits Npad columns further: one FP32 sum per item
                            float u[8];
                            tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(lt * tstride + Npad + c8), u);
#pragma unroll
                            for (int i = 0; i < 8; ++i) v[i] = __fadd_rn(v[i], u[i]);
                        }
                        if (!valid) continue;
                        const int wsel = c8 >> 5;
                        const unsigned wm = __ldg(&pp->mask[wsel]);
                        const unsigned w = (wm >> (c8 & 31)) & 0xffu;
                        if (!w) continue;
                        int idx = __ldg(&pp->first) - it0 + __popc(wm & ((1u << (c8 & 31)) - 1u));
                        for (int m = 0; m < wsel; ++m) idx += __popc(__ldg(&pp->mask[m]));
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if ((w >> i) & 1u) kahan_add(sums[idx++], v[i]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.accf);
            ++nfl;
        };
        for (long long ci = c0; ci < c1; ++ci) {
            role_wait(&bars.sfull[rs.slot], rs.phase, abortp, err, 20, wait_limit);
            const unsigned char *st = stg + rs.slot * stage_bytes;
            if constexpr (BW == 0) {
                // ---- operand B: split every inner row into BF16 hi/lo (swizzled K-major)
                const int sb = rb.slot;
                if (rb.warm) role_wait(&bars.bempty[sb], rb.phase ^ 1u, abortp, err, 21, wait_limit);
                build_b<AW, KA>(st, half_bytes, s_inner, nbuild, warp, lane, Bh0 + 2 * sb * b_stage,
                                Bh0 + 2 * sb * b_stage + b_tile, b_atom2);
                if (!bfa) {  // else operand B is complete once the pair products below are stored
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bars.bfull[sb]);
                    rb.next();
                }
            }
            // ---- operand A: pair products of this thread's row, PPT points, into TMEM
            for (int lt = 0; lt < ntl; ++lt) {
                const int as = ra.slot;
                if (ra.warm) role_wait(&bars.empty[as], ra.phase ^ 1u, abortp, err, 22, wait_limit);
                tc_fence_after();
                if (!idle) {
                    const int2 bc = pbc[lt * 128 + (stacked ? (r & 63) : r)];
                    const uint32_t lanebase = tmem + ((uint32_t)(32 * q) << 16);
                    const uint32_t col = (uint32_t)(acc_cols + as * ACOLS + (PPT / 2) * kq);
                    // This thread's 16-byte chunks of the step are J0 + k, k < PPT / 4,
                    // J0 = (PPT/4) kq a multiple of 4 that never carries into the next
                    // 32-point box.  The stage row of bin b holds chunk J at
                    // ((J & 7) ^ (b & 7)) << 4 of box J >> 3, so every address is the
                    // row's base XOR a compile-time offset.
                    const int J0 = (PPT / 4) * kq;
                    const unsigned char *rb0 = st + (J0 >> 3) * half_bytes + (bc.x >= 0 ? bc.x : 0) * 128;
                    const unsigned char *rc0 = st + (J0 >> 3) * half_bytes + (bc.y >= 0 ? bc.y : 0) * 128;
                    const uint32_t xb = (uint32_t)(((bc.x & 7) ^ (J0 & 7)) << 4);
                    const uint32_t xc = (uint32_t)(((bc.y & 7) ^ (J0 & 7)) << 4);
                    // 16 points (8 columns of hi, 8 of lo) at a time
#pragma unroll
                    for (int c = 0; c < PPT / 16; ++c) {
                        uint32_t hw[8], lw[8];
                        if (bc.x >= 0) {
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
                                const uint32_t k0 = (uint32_t)((4 * c + 2 * j) << 4), k1 = k0 + 16u;
                                const float4 b0 = *reinterpret_cast<const float4 *>(rb0 + (k0 ^ xb));
                                const float4 b1 = *reinterpret_cast<const float4 *>(rb0 + (k1 ^ xb));
                                const float4 e0 = *reinterpret_cast<const float4 *>(rc0 + (k0 ^ xc));
                                const float4 e1 = *reinterpret_cast<const float4 *>(rc0 + (k1 ^ xc));
                                mul_split8(b0, b1, e0, e1, hw + 4 * j, lw + 4 * j);
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 8; ++j) hw[j] = lw[j] = 0u;
                        }
                        if (!stacked) {
                            tmem_st8a(lanebase + col + 8u * c, hw);
                            tmem_st8a(lanebase + col + 32u * KA + 8u * c, lw);
                        } else if (q < 2) {  // stacked: the hi words in rows 0..63, the lo words in 64..127
                            tmem_st8a(lanebase + col + 8u * c, hw);
                        } else {
                            tmem_st8a(lanebase + col + 8u * c, lw);
                        }
                        if (FEED && feed >= 0) {
                            // the same product is inner row `feed`: its 8-point groups
                            // PPT kq / 8 + 2c (hw[0..3]) and + 1 (hw[4..7]) go to operand B
                            unsigned char *bh = Bh0 + 2 * rb.slot * b_stage;
#pragma unroll
                            for (int h2 = 0; h2 < 2; ++h2) {
                                const int u = (PPT / 8) * kq + 2 * c + h2;
                                const uint32_t off = (uint32_t)((u >> 3) * b_atom2) + sw128_off(feed, u & 7);
                                *reinterpret_cast<uint4 *>(bh + off) =
                                    make_uint4(hw[4 * h2], hw[4 * h2 + 1], hw[4 * h2 + 2], hw[4 * h2 + 3]);
                                *reinterpret_cast<uint4 *>(bh + b_tile + off) =
                                    make_uint4(lw[4 * h2], lw[4 * h2 + 1], lw[4 * h2 + 2], lw[4 * h2 + 3]);
                            }
                        }
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                }
                tc_fence_before();
                if (FEED) fence_proxy_async_smem();  // operand B's stores, for the MMAs
                __syncwarp();
                if (lane == 0) {
                    if (FEED) mbar_arrive(&bars.bfull[rb.slot]);
                    mbar_arrive(&bars.full[as]);
                }
                if (FEED) rb.next();
                ra.next();
            }
            // ---- the stage is consumed: hand it back to the loader
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.sempty[rs.slot]);
            rs.next();
            // ---- flush: accumulators -> compensated FP32 sums.  A flush point's
            // flush runs after the next step's operands are handed off (the MMAs
            // of that step wait for it), so forming them overlaps the drain of
            // the MMAs before the flush point.  Only when a step's tiles fit in
            // the A ring (ntl <= NST): their stages are then freed by MMAs of
            // steps before the flush point, never by the next step's own MMAs,
            // which wait for the flush.  The last step flushes at once.
            const bool point = ++since == flush_every || ci == c1 - 1;
            if (pend) {
                flush();
                pend = false;
            }
            if (point) {
                since = 0;
                if (ci == c1 - 1 || ntl > NST) flush();
                else pend = true;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    double *row = part + ((long long)blockIdx.z * part_rows + blockIdx.x) * nitems_total;
    for (int i = tid; i < nloc; i += kTcThreads)
        row[iout[it0 + i]] += ((double)acc[i].x - (double)acc[i].y) +
                              (stacked ? (double)acc2[i].x - (double)acc2[i].y : 0.0);
}


// ======================================================================
// Wide orientation.  The per-instruction cost of tcgen05.mma barely grows
// with N up to 256 (measured ~130-145 cycles for N = 64..256, M = 128,
// K = 16), so the operand with the most rows goes to N:
//   operand A (M = 128, tensor memory): up to 64 "left" rows stacked as
//       [hi; lo] -- the single bins a (bispectrum) or the outer pairs (c, d)
//       (trispectrum) -- written once per chunk;
//   operand B (N <= 256, shared memory): the "right" pair products
//       (b, c) (bispectrum) or inner pairs (a, b) (trispectrum), split hi/lo;
//   D[row][right] accumulates hi*(Phi + Plo) in rows 0..63 and
//   lo*(Phi + Plo) in rows 64..127: every product of the two splits (BF16x4).
// Groups of 256 right rows go to different CTA rows of the grid.
// ======================================================================

constexpr int kWideN = 256;
constexpr int kWideAcol = 256;  // TMEM column of the A stages (after D)

struct WideBars {
    uint64_t full[2], empty[2], accr, accf;
};

constexpr int kWideProd = 16;  // producer warps of the wide kernel (4 per TMEM lane quarter)
constexpr int kWideThreads = (kWideProd + 1) * 32;

__device__ __forceinline__ void tmem_st8w(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
        "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
        : "memory");
}

__global__ void __launch_bounds__(kWideThreads, 1)
    contract_wide_kernel(const float *__restrict__ I, long long bin_stride, long long npts, int nbins,
                         int nleft, const int2 *__restrict__ left, const WideRight *__restrict__ rights,
                         int nright, const int *__restrict__ item_out, int nitems_total,
                         double *__restrict__ part, int x4, int flush_every, int *__restrict__ err,
                         long long wait_limit) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ WideBars bars;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int2 s_left[64];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.y * kWideN;
    const int cnt = min(kWideN, nright - r0);
    const int Ng = ((cnt + 15) / 16) * 16;

    uintptr_t base = (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023;
    unsigned char *sm = reinterpret_cast<unsigned char *>(base);
    const int b_tile = kWideN * 128;
    unsigned char *const Bh0 = sm, *const Bl0 = sm + 2 * b_tile;
    float *stage = reinterpret_cast<float *>(sm + 4 * b_tile);
    const int stage_floats = nbins * kStageLd;
    const int ncols = 512;
    // items of this group: FP32 per-flush sums, one per (item, row half): no
    // two threads ever add to the same word, so the result is deterministic
    const int first0 = rights[r0].first;
    const int nloc = rights[r0 + cnt - 1].first + __popcll(rights[r0 + cnt - 1].mask) - first0;
    float *acc32 = stage + 2 * stage_floats;                       // [2][nloc]
    WideRight *s_r = reinterpret_cast<WideRight *>(acc32 + ((2 * nloc + 3) & ~3));

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bars.full[i], kWideProd);
            mbar_init(&bars.empty[i], 1);
        }
        mbar_init(&bars.accr, 1);
        mbar_init(&bars.accf, kWideProd);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == kWideProd) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < 64; i += kWideThreads) s_left[i] = i < nleft ? left[i] : make_int2(-1, -1);
    for (int i = tid; i < 2 * nloc; i += kWideThreads) acc32[i] = 0.f;
    for (int i = tid; i < cnt; i += kWideThreads) s_r[i] = rights[r0 + i];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abortp = &abort_flag;

    const long long nchunks = (npts + KC - 1) / KC;
    const long long c0 = nchunks * blockIdx.x / gridDim.x;
    const long long c1 = nchunks * (blockIdx.x + 1) / gridDim.x;
    double *prow = part + (long long)blockIdx.x * nitems_total;

    if (warp == kWideProd) {
        // ================= MMA issuer =================
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, Ng);
            long long g = 0, nfl = 0;
            bool fresh = true;
            int since = 0;
            for (long long ci = c0; ci < c1; ++ci) {
                const int s = (int)(g & 1);
                const bool ok = role_wait(&bars.full[s], (uint32_t)((g >> 1) & 1), abortp, err, 31, wait_limit);
                tc_fence_after();
                if (ok && !*abortp) {
                    const uint32_t a = tmem + (uint32_t)(kWideAcol + 32 * s);
                    const uint64_t dh = sdesc_sw128(smem_u32(Bh0 + s * b_tile));
                    const uint64_t dl = sdesc_sw128(smem_u32(Bl0 + s * b_tile));
                    if (fresh) mma_ts<false>(tmem, a, dh, idesc);
                    else mma_ts<true>(tmem, a, dh, idesc);
                    if (x4) mma_ts<true>(tmem, a, dl, idesc);
#pragma unroll
                    for (int k = 1; k < 4; ++k) {
                        mma_ts<true>(tmem, a + 8u * k, dh + 2u * k, idesc);
                        if (x4) mma_ts<true>(tmem, a + 8u * k, dl + 2u * k, idesc);
                    }
                }
                mma_commit(&bars.empty[s]);
                ++g;
                fresh = false;
                if (++since == flush_every || ci == c1 - 1) {
                    mma_commit(&bars.accr);
                    role_wait(&bars.accf, (uint32_t)(nfl & 1), abortp, err, 32, wait_limit);
                    tc_fence_after();
                    ++nfl;
                    fresh = true;
                    since = 0;
                }
            }
            if (g > 0) {
                const int s = (int)((g - 1) & 1);
                if (!mbar_wait(&bars.empty[s], (uint32_t)(((g - 1) >> 1) & 1))) atomicExch(err, 34);
            }
        }
    } else {
        // ================= producers (warps 0..15) =================
        const int ptid = tid;
        constexpr int NP = kWideProd * 32;
        const int q = warp & 3, kq = warp >> 2;  // TMEM lane quarter; 16-point slice of the chunk
        const int r = 32 * q + lane;             // operand-A row written by this thread
        const int li = r & 63, half = r >> 6;
        auto prefetch = [&](long long ch, int s) {
            const long long q0 = ch * KC;
            float *dst = stage + s * stage_floats;
            for (int i = ptid; i < nbins * (KC / 4); i += NP) {
                int b = i / (KC / 4), k4 = i - b * (KC / 4);
                long long qq = q0 + 4LL * k4;
                long long rem = npts - qq;
                int bytes = rem >= 4 ? 16 : (rem > 0 ? (int)rem * 4 : 0);
                const float *src = bytes ? (I + b * bin_stride + qq) : I;
                cp_async16(smem_u32(dst + b * kStageLd + 4 * k4), src, bytes);
            }
            cp_async_commit();
        };
        long long g = 0, nfl = 0;
        int since = 0;
        if (c0 < c1) prefetch(c0, 0);
        for (long long ci = c0; ci < c1; ++ci) {
            const int s = (int)(g & 1);
            cp_async_wait_all();
            asm volatile("bar.sync 1, %0;" ::"n"(NP) : "memory");
            if (ci + 1 < c1) prefetch(ci + 1, s ^ 1);
            const float *st = stage + s * stage_floats;
            if (g >= 2) role_wait(&bars.empty[s], (uint32_t)(((g - 2) >> 1) & 1), abortp, err, 41, wait_limit);
            tc_fence_after();
            // ---- operand A: left row li, points 16kq .. 16kq+15, hi (rows 0..63) or lo (64..127)
            {
                uint32_t words[8];
                const int2 lf = s_left[li];
                if (lf.x >= 0 && (half == 0 || x4)) {
#pragma unroll
                    for (int jj = 0; jj < 2; ++jj) {
                        const int j = 2 * kq + jj;
                        const float4 *ra = reinterpret_cast<const float4 *>(st + lf.x * kStageLd + 8 * j);
                        float4 a0 = ra[0], a1 = ra[1];
                        if (lf.y >= 0) {
                            const float4 *rb = reinterpret_cast<const float4 *>(st + lf.y * kStageLd + 8 * j);
                            float4 b0 = rb[0], b1 = rb[1];
                            a0 = make_float4(a0.x * b0.x, a0.y * b0.y, a0.z * b0.z, a0.w * b0.w);
                            a1 = make_float4(a1.x * b1.x, a1.y * b1.y, a1.z * b1.z, a1.w * b1.w);
                        }
                        float v[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                        uint4 h, l;
                        split8(v, h, l);
                        const uint4 o = half ? l : h;
                        words[4 * jj + 0] = o.x; words[4 * jj + 1] = o.y;
                        words[4 * jj + 2] = o.z; words[4 * jj + 3] = o.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) words[j] = 0u;
                }
                tmem_st8w(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kWideAcol + 32 * s + 8 * kq), words);
            }
            // ---- operand B: right pair products, hi and lo, swizzled K-major
            for (int u = ptid; u < Ng * 8; u += NP) {
                const int rr = u % Ng, j = u / Ng;
                uint4 h = make_uint4(0, 0, 0, 0), l = make_uint4(0, 0, 0, 0);
                if (rr < cnt) {
                    const int2 xy = *reinterpret_cast<const int2 *>(&s_r[rr]);
                    const float4 *rb = reinterpret_cast<const float4 *>(st + xy.x * kStageLd + 8 * j);
                    const float4 *rc = reinterpret_cast<const float4 *>(st + xy.y * kStageLd + 8 * j);
                    float4 b0 = rb[0], b1 = rb[1], e0 = rc[0], e1 = rc[1];
                    float v[8] = {b0.x * e0.x, b0.y * e0.y, b0.z * e0.z, b0.w * e0.w,
                                  b1.x * e1.x, b1.y * e1.y, b1.z * e1.z, b1.w * e1.w};
                    split8(v, h, l);
                }
                const uint32_t off = sw128_off(rr, j);
                *reinterpret_cast<uint4 *>(Bh0 + s * b_tile + off) = h;
                *reinterpret_cast<uint4 *>(Bl0 + s * b_tile + off) = l;
            }
            fence_proxy_async_smem();
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.full[s]);
            ++g;
            // ---- flush: D -> FP32 shared sums of (item, half)
            if (++since == flush_every || ci == c1 - 1) {
                role_wait(&bars.accr, (uint32_t)(nfl & 1), abortp, err, 42, wait_limit);
                tc_fence_after();
                if (!*abortp) {
                    const unsigned long long lbit = 1ULL << li;
                    float *a32 = acc32 + half * nloc;
                    for (int c8 = 8 * kq; c8 < Ng; c8 += 32) {
                        float v[8];
                        tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c8, v);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int rr = c8 + i;
                            if (rr >= cnt) continue;
                            const unsigned long long m = s_r[rr].mask;
                            if (!(m & lbit)) continue;
                            a32[s_r[rr].first - first0 + __popcll(m & (lbit - 1ULL))] += v[i];
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars.accf);
                ++nfl;
                since = 0;
                // every 8 flushes (and at the end) add the FP32 sums to the FP64 row
                if ((nfl & 7) == 0 || ci == c1 - 1) {
                    asm volatile("bar.sync 1, %0;" ::"n"(NP) : "memory");
                    for (int i = ptid; i < nloc; i += NP) {
                        prow[item_out[first0 + i]] += (double)acc32[i] + (double)acc32[nloc + i];
                        acc32[i] = 0.f;
                        acc32[nloc + i] = 0.f;
                    }
                    asm volatile("bar.sync 1, %0;" ::"n"(NP) : "memory");
                }
            }
        }
        cp_async_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kWideProd)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ------------------------------------------------------------------ host side
// Dynamic shared memory of the narrow kernel: B tiles, nstg field stages,
// compensated sums, pair bins.
static size_t tc_smem_bytes(int nbins, int Npad, int nloc, int ntl, int nstg, int ka = 1, int nsb = 2) {
    const size_t half = (size_t)((nbins + 7) & ~7) * 128;
    size_t b = 1024 + 2 * (size_t)nsb * ka * Npad * 128 + (size_t)nstg * 2 * ka * half + (size_t)nloc * 8 +
               (size_t)ntl * 128 * 8;
    return std::max<size_t>(b, 116 * 1024);  // > half the SM's shared memory: one CTA per SM
}

static int tile_stride(int Npad) { return ((Npad + 31) / 32) * 32; }

// Hand-off wait limit of the plan's launches (FBS_OPT_TC_WAIT_LIMIT; 0 = the default).
static long long tc_wait_limit(const Plan &p) { return p.tc_wait_limit > 0 ? p.tc_wait_limit : kWaitCycles; }

static TcState &tc_state(Plan &p) {
    if (!p.tc) {
        TcState *st = new TcState();
        p.tc = st;
        st->d_err = p.root().d_errbuf;
    }
    return *reinterpret_cast<TcState *>(p.tc);
}

// Group the pair tiles of a job (tensor memory and the compensated item sums
// bound a group) and upload its tables.  hp: outer pairs (masks, first item),
// inner: inner rows, iout: output column of every item in job order.
static void finish_job(Plan &p, TcJob &job, const std::vector<TcPair> &hp, const std::vector<int2> &inner,
                       const std::vector<int> &iout) {
    job.npairs = (int)hp.size();
    job.ntiles = (job.npairs + 127) / 128;
    job.ninner = (int)inner.size();
    if (job.ninner > kMaxInner || job.npairs == 0) return;  // not usable on the tensor cores
    job.Npad = std::max(16, ((job.ninner + 15) / 16) * 16);
    auto items_of = [&](int pa, int pe) {
        int n = 0;
        for (int i = pa; i < pe; ++i)
            for (int w = 0; w < kMaxInner / 32; ++w) n += __builtin_popcount(hp[i].mask[w]);
        return n;
    };
    const size_t smem_cap = 220 * 1024;
    job.grp.assign(1, 0);
    int cur_tiles = 0, cur_items = 0;
    job.maxloc = 0;
    for (int tt = 0; tt < job.ntiles; ++tt) {
        int pa = tt * 128, pe = std::min(job.npairs, pa + 128);
        int items = items_of(pa, pe);
        const int acc_cols = (((cur_tiles + 1) * tile_stride(job.Npad) + 31) / 32) * 32;
        bool fits = acc_cols + 2 * kAStageCols <= 512 &&
                    tc_smem_bytes(p.nbins, job.Npad, cur_items + items, cur_tiles + 1, 2) <= smem_cap;
        if (cur_tiles > 0 && !fits) {
            job.grp.push_back(tt);
            job.maxloc = std::max(job.maxloc, cur_items);
            cur_tiles = 0;
            cur_items = 0;
        }
        cur_tiles += 1;
        cur_items += items;
    }
    job.maxloc = std::max(job.maxloc, cur_items);
    job.grp.push_back(job.ntiles);
    job.maxtiles = 0;
    for (size_t gi = 0; gi + 1 < job.grp.size(); ++gi)
        job.maxtiles = std::max(job.maxtiles, job.grp[gi + 1] - job.grp[gi]);
    if (p.nbins > 256) return;  // one TMA box spans every bin
    if (tc_smem_bytes(p.nbins, job.Npad, job.maxloc, job.maxtiles, 2) > smem_cap) return;
    if ((((job.maxtiles * tile_stride(job.Npad)) + 31) / 32) * 32 + 2 * kAStageCols > 512) return;
    job.d_pairs = (TcPair *)p.dalloc(hp.size() * sizeof(TcPair));
    FBS_CUDA(cudaMemcpyAsync(job.d_pairs, hp.data(), hp.size() * sizeof(TcPair), cudaMemcpyHostToDevice,
                             p.stream));
    job.d_inner = (int2 *)p.dalloc(inner.size() * sizeof(int2));
    FBS_CUDA(cudaMemcpyAsync(job.d_inner, inner.data(), inner.size() * sizeof(int2), cudaMemcpyHostToDevice,
                             p.stream));
    job.d_iout = (int *)p.dalloc(std::max<size_t>(1, iout.size()) * sizeof(int));
    FBS_CUDA(cudaMemcpyAsync(job.d_iout, iout.data(), iout.size() * sizeof(int), cudaMemcpyHostToDevice,
                             p.stream));
    job.d_grp = (int *)p.dalloc(job.grp.size() * sizeof(int));
    FBS_CUDA(cudaMemcpyAsync(job.d_grp, job.grp.data(), job.grp.size() * sizeof(int),
                             cudaMemcpyHostToDevice, p.stream));
    FBS_CUDA(cudaStreamSynchronize(p.stream));  // host tables go out of scope
    job.usable = true;
}

// Bispectrum job with every triplet (a <= b <= c) carried by one of its three
// pairs: sum_x I_a I_b I_c is the same whichever two fields form the product
// and which one is the inner row.  A greedy set cover (the pair that carries
// the most uncovered triplets first, ties to the smaller pair) keeps the
// outer rows, and so the 128-row tiles, few: 378 instead of 546 pairs for 64
// log bins at 512^3.
static void build_covered_job(Plan &p, const TaskList &t, TcJob &job) {
    const int nb = p.nbins;
    std::vector<std::array<int, 3>> trip;
    std::vector<int> out;
    for (int i = 0; i < t.npairs; ++i)
        for (int e = t.pstart[i]; e < t.pstart[i + 1]; ++e) {
            std::array<int, 3> tr = {t.ia[e], t.pb[i], t.pc[i]};
            std::sort(tr.begin(), tr.end());
            trip.push_back(tr);
            out.push_back(t.iout[e]);
        }
    const int T = (int)trip.size();
    const std::vector<int> assigned = cover_triplet_pairs(nb, trip);
    // outer rows in pair order; items of a row: the remaining bin, ascending
    std::map<int, std::vector<std::pair<int, int>>> rows;  // pair key -> (inner bin, output)
    for (int i = 0; i < T; ++i) {
        const int x = assigned[i] / nb, y = assigned[i] % nb;
        std::array<int, 3> rest = trip[i];
        auto it = std::find(rest.begin(), rest.end(), x);
        *it = -1;
        it = std::find(rest.begin(), rest.end(), y);
        *it = -1;
        int z = -1;
        for (int v : rest) if (v >= 0) z = v;
        rows[assigned[i]].push_back({z, out[i]});
    }
    std::vector<int2> inner;
    for (int b = 0; b < nb; ++b) inner.push_back(make_int2(b, -1));
    std::vector<TcPair> hp;
    std::vector<int> iout;
    for (auto &kv : rows) {
        auto &items = kv.second;
        std::sort(items.begin(), items.end());
        TcPair q{};
        q.b = kv.first / nb;
        q.c = kv.first % nb;
        q.first = (int)iout.size();
        int prev = -1;
        for (auto &it : items) {
            if (it.first <= prev) throw Failure{FBS_ERR_ARG, "pair cover: repeated inner bin"};
            prev = it.first;
            q.mask[it.first >> 5] |= 1u << (it.first & 31);
            iout.push_back(it.second);
        }
        hp.push_back(q);
    }
    finish_job(p, job, hp, inner, iout);
}

// One contraction from its pair-grouped task list: inner rows are the single
// bins (bispectrum) or the distinct inner pairs (trispectrum).
static void build_job(Plan &p, const TaskList &t, bool quads, TcJob &job) {
    job.built = true;
    job.variant = quads ? 0 : p.tc_pairs;
    if (!quads && p.tc_pairs == 0 && p.nbins <= kMaxInner) {
        build_covered_job(p, t, job);
        return;
    }
    std::vector<int2> inner;
    std::vector<int> row_of;  // (a, b) -> inner row, a*nbins+b
    if (!quads) {
        for (int b = 0; b < p.nbins; ++b) inner.push_back(make_int2(b, -1));
    } else {
        row_of.assign((size_t)p.nbins * p.nbins, -1);
        for (int e = 0; e < t.nitems; ++e) row_of[(size_t)t.ia[e] * p.nbins + t.ib[e]] = 0;
        for (int a = 0; a < p.nbins; ++a)
            for (int b = 0; b < p.nbins; ++b)
                if (row_of[(size_t)a * p.nbins + b] >= 0) {
                    row_of[(size_t)a * p.nbins + b] = (int)inner.size();
                    inner.push_back(make_int2(a, b));
                }
    }
    if ((int)inner.size() > kMaxInner) return;
    std::vector<TcPair> hp(t.npairs);
    for (int i = 0; i < t.npairs; ++i) {
        TcPair q{};
        q.b = t.pb[i];
        q.c = t.pc[i];
        q.first = t.pstart[i];
        int prev = -1;
        for (int e = t.pstart[i]; e < t.pstart[i + 1]; ++e) {
            int n = quads ? row_of[(size_t)t.ia[e] * p.nbins + t.ib[e]] : t.ia[e];
            if (n <= prev) throw Failure{FBS_ERR_ARG, "tensor-core task list not sorted by inner row"};
            prev = n;
            q.mask[n >> 5] |= 1u << (n & 31);
        }
        hp[i] = q;
    }
    finish_job(p, job, hp, inner, t.iout);
}

// A job with a single pair tile whose inner rows from nbuild on are pair
// rows that are outer rows too (the same product I_x I_y): the operand-A
// thread of such an outer row also stores the row's BF16 hi/lo values into
// operand B, and only inner rows 0..nbuild-1 are built from the field stage.
// The products are the same FP32 multiplications, so the sums are
// bit-identical.
static void attach_feed(Plan &p, TcJob &job, const std::vector<TcPair> &hp, const std::vector<int2> &inner,
                        int nbuild) {
    if (job.ntiles != 1 || nbuild >= (int)inner.size()) return;
    std::map<std::pair<int, int>, int> outer_row;
    for (int i = 0; i < (int)hp.size(); ++i)
        outer_row.emplace(std::make_pair(std::min(hp[i].b, hp[i].c), std::max(hp[i].b, hp[i].c)), i);
    std::vector<int> feed(128, -1);
    for (int n = nbuild; n < (int)inner.size(); ++n) {
        if (inner[n].y < 0) return;
        auto it = outer_row.find({std::min(inner[n].x, inner[n].y), std::max(inner[n].x, inner[n].y)});
        if (it == outer_row.end() || feed[it->second] >= 0) return;
        feed[it->second] = n;
    }
    job.nsingle = nbuild;
    job.d_ifeed = (int *)p.dalloc(feed.size() * sizeof(int));
    FBS_CUDA(cudaMemcpyAsync(job.d_ifeed, feed.data(), feed.size() * sizeof(int), cudaMemcpyHostToDevice,
                             p.stream));
    FBS_CUDA(cudaStreamSynchronize(p.stream));
}

// The triplets and quadruplets of a trispectrum plan as one contraction over
// the same shell fields: outer rows are the union of the triplets' pairs
// (b, c) and the quadruplets' pairs (c, d); inner rows are the triplets'
// single bins a followed by the quadruplets' inner pairs (a, b).  Output
// column of a triplet: its index; of a quadruplet: ntrip + its index.
static void build_fused_job(Plan &p, TcJob &job) {
    job.built = true;
    job.variant = p.tc_pairs;
    const TaskList &tt = p.ttask, &qt = p.qtask;
    const int nb = p.nbins;
    // (inner pair, outer pair) of every quadruplet item, in task order
    std::vector<std::pair<int, int>> qassign(qt.nitems);
    for (int i = 0; i < qt.npairs; ++i)
        for (int e = qt.pstart[i]; e < qt.pstart[i + 1]; ++e)
            qassign[e] = {qt.ia[e] * nb + qt.ib[e], qt.pb[i] * nb + qt.pc[i]};
    if (p.tc_pairs == 0) {
        std::vector<std::array<int, 4>> quads(qt.nitems);
        for (int i = 0; i < qt.npairs; ++i)
            for (int e = qt.pstart[i]; e < qt.pstart[i + 1]; ++e) {
                quads[e] = {qt.ia[e], qt.ib[e], qt.pb[i], qt.pc[i]};
                std::sort(quads[e].begin(), quads[e].end());
            }
        std::vector<int> fixed;
        for (int i = 0; i < tt.npairs; ++i) fixed.push_back(tt.pb[i] * nb + tt.pc[i]);
        std::vector<std::pair<int, int>> a;
        if (cover_quad_pairings(nb, quads, fixed, a)) qassign = a;
    }
    std::vector<int> bin_row(nb, -1), pair_row((size_t)nb * nb, -1);
    for (int e = 0; e < tt.nitems; ++e) bin_row[tt.ia[e]] = 0;
    for (int e = 0; e < qt.nitems; ++e) pair_row[qassign[e].first] = 0;
    // outer rows (unordered pairs); an inner pair that is an outer row too is
    // "fed" (operand A forms its product).  While one tile holds them all,
    // the other inner pairs join the outer rows without items.
    std::vector<char> is_outer((size_t)nb * nb, 0);
    auto mark = [&](int x, int y) { is_outer[(size_t)std::min(x, y) * nb + std::max(x, y)] = 1; };
    size_t nouter = 0;
    for (int i = 0; i < tt.npairs; ++i) mark(tt.pb[i], tt.pc[i]);
    for (int e = 0; e < qt.nitems; ++e) mark(qassign[e].second / nb, qassign[e].second % nb);
    for (char c : is_outer) nouter += c;
    std::vector<std::pair<int, int>> extra;
    auto fed = [&](int a, int b) { return is_outer[(size_t)std::min(a, b) * nb + std::max(a, b)] != 0; };
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b)
            if (pair_row[(size_t)a * nb + b] >= 0 && !fed(a, b)) extra.push_back({std::min(a, b), std::max(a, b)});
    std::sort(extra.begin(), extra.end());
    extra.erase(std::unique(extra.begin(), extra.end()), extra.end());
    const bool add_extra = nouter + extra.size() <= 128;
    if (add_extra)
        for (const auto &k : extra) mark(k.first, k.second);
    // inner rows: single bins, then the pairs built from the field stage, then
    // the fed pairs in the order of their outer rows (the outer rows are the
    // keys of `outer` below in ascending order), so that the operand-A lanes
    // of a warp store consecutive inner rows (distinct swizzle positions)
    std::set<std::pair<int, int>> okeys;
    for (int i = 0; i < tt.npairs; ++i) okeys.insert({tt.pb[i], tt.pc[i]});
    for (int e = 0; e < qt.nitems; ++e) okeys.insert({qassign[e].second / nb, qassign[e].second % nb});
    if (add_extra)
        for (const auto &k : extra)
            if (!okeys.count(k) && !okeys.count({k.second, k.first})) okeys.insert(k);
    std::vector<int2> inner;
    for (int b = 0; b < nb; ++b)
        if (bin_row[b] >= 0) {
            bin_row[b] = (int)inner.size();
            inner.push_back(make_int2(b, -1));
        }
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b)
            if (pair_row[(size_t)a * nb + b] >= 0 && !fed(a, b)) {
                pair_row[(size_t)a * nb + b] = (int)inner.size();
                inner.push_back(make_int2(a, b));
            }
    {
        std::vector<std::pair<int, int>> fed_pairs;  // (outer rank, a * nb + b)
        for (int a = 0; a < nb; ++a)
            for (int b = 0; b < nb; ++b)
                if (pair_row[(size_t)a * nb + b] >= 0 && fed(a, b)) {
                    auto it = okeys.find({a, b});
                    if (it == okeys.end()) it = okeys.find({b, a});
                    fed_pairs.push_back({it == okeys.end() ? (int)okeys.size()
                                                           : (int)std::distance(okeys.begin(), it),
                                         a * nb + b});
                }
        std::sort(fed_pairs.begin(), fed_pairs.end());
        for (const auto &f : fed_pairs) {
            pair_row[(size_t)f.second] = (int)inner.size();
            inner.push_back(make_int2(f.second / nb, f.second % nb));
        }
    }
    int nbuild = 0;
    while (nbuild < (int)inner.size() && (inner[nbuild].y < 0 || !fed(inner[nbuild].x, inner[nbuild].y))) ++nbuild;
    if ((int)inner.size() > kMaxInner) return;
    std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> outer;  // (x, y) -> (inner row, column)
    for (int i = 0; i < tt.npairs; ++i)
        for (int e = tt.pstart[i]; e < tt.pstart[i + 1]; ++e)
            outer[{tt.pb[i], tt.pc[i]}].push_back({bin_row[tt.ia[e]], tt.iout[e]});
    for (int e = 0; e < qt.nitems; ++e)
        outer[{qassign[e].second / nb, qassign[e].second % nb}].push_back({pair_row[qassign[e].first],
                                                                          tt.nitems + qt.iout[e]});
    if (add_extra)
        for (const auto &k : extra)
            if (!outer.count(k) && !outer.count({k.second, k.first})) outer[k];
    std::vector<TcPair> hp;
    std::vector<int> iout;
    hp.reserve(outer.size());
    iout.reserve((size_t)tt.nitems + qt.nitems);
    for (auto &kv : outer) {
        auto &items = kv.second;
        std::sort(items.begin(), items.end());
        TcPair q{};
        q.b = kv.first.first;
        q.c = kv.first.second;
        q.first = (int)iout.size();
        int prev = -1;
        for (auto &it : items) {
            if (it.first <= prev) throw Failure{FBS_ERR_ARG, "fused contraction: repeated item"};
            prev = it.first;
            q.mask[it.first >> 5] |= 1u << (it.first & 31);
            iout.push_back(it.second);
        }
        hp.push_back(q);
    }
    finish_job(p, job, hp, inner, iout);
    if (job.usable)
        p.d_fpart = (double *)p.dalloc((size_t)p.part_blocks * (tt.nitems + qt.nitems) * sizeof(double));
    if (job.usable) attach_feed(p, job, hp, inner, nbuild);
}

// Wide orientation tables: left rows (<= 64), right rows, items ordered by
// (right, left) with their output indices.
static void build_wide(Plan &p, bool quads, WideJob &w) {
    w.built = true;
    const TaskList &t = quads ? p.qtask : p.ttask;
    if (t.nitems == 0) return;
    std::vector<int2> left;
    std::vector<int2> rightbins;
    // (right, left, out) triples
    std::vector<std::array<int, 3>> it;
    if (!quads) {
        // left = single bins a; right = outer pairs (b, c)
        for (int b = 0; b < p.nbins; ++b) left.push_back(make_int2(b, -1));
        for (int i = 0; i < t.npairs; ++i) rightbins.push_back(make_int2(t.pb[i], t.pc[i]));
        for (int i = 0; i < t.npairs; ++i)
            for (int e = t.pstart[i]; e < t.pstart[i + 1]; ++e) it.push_back({i, t.ia[e], t.iout[e]});
    } else {
        // left = outer pairs (c, d); right = distinct inner pairs (a, b)
        for (int i = 0; i < t.npairs; ++i) left.push_back(make_int2(t.pb[i], t.pc[i]));
        std::vector<int> ridx((size_t)p.nbins * p.nbins, -1);
        for (int e = 0; e < t.nitems; ++e) ridx[t.ia[e] * p.nbins + t.ib[e]] = 0;
        for (int a = 0; a < p.nbins; ++a)
            for (int b = 0; b < p.nbins; ++b)
                if (ridx[a * p.nbins + b] >= 0) {
                    ridx[a * p.nbins + b] = (int)rightbins.size();
                    rightbins.push_back(make_int2(a, b));
                }
        for (int i = 0; i < t.npairs; ++i)
            for (int e = t.pstart[i]; e < t.pstart[i + 1]; ++e)
                it.push_back({ridx[t.ia[e] * p.nbins + t.ib[e]], i, t.iout[e]});
    }
    if ((int)left.size() > 64) return;  // the narrow kernel handles it
    std::sort(it.begin(), it.end());
    std::vector<WideRight> R(rightbins.size());
    for (size_t i = 0; i < rightbins.size(); ++i) {
        R[i] = WideRight{rightbins[i].x, rightbins[i].y, 0, 0, 0ULL};
    }
    std::vector<int> out(it.size());
    int prev_r = -1;
    for (size_t k = 0; k < it.size(); ++k) {
        const int r = it[k][0], l = it[k][1];
        if (r != prev_r) {
            R[r].first = (int)k;
            prev_r = r;
        }
        R[r].mask |= 1ULL << l;
        out[k] = it[k][2];
    }
    w.nleft = (int)left.size();
    w.nright = (int)R.size();
    w.nitems = (int)it.size();
    for (int r0 = 0; r0 < w.nright; r0 += kWideN) {
        const int r1 = std::min(w.nright, r0 + kWideN) - 1;
        const int n = R[r1].first + __builtin_popcountll(R[r1].mask) - R[r0].first;
        w.maxloc = std::max(w.maxloc, n);
    }
    w.d_left = (int2 *)p.dalloc(left.size() * sizeof(int2));
    FBS_CUDA(cudaMemcpyAsync(w.d_left, left.data(), left.size() * sizeof(int2), cudaMemcpyHostToDevice, p.stream));
    w.d_rights = (WideRight *)p.dalloc(R.size() * sizeof(WideRight));
    FBS_CUDA(cudaMemcpyAsync(w.d_rights, R.data(), R.size() * sizeof(WideRight), cudaMemcpyHostToDevice, p.stream));
    w.d_item_out = (int *)p.dalloc(out.size() * sizeof(int));
    FBS_CUDA(cudaMemcpyAsync(w.d_item_out, out.data(), out.size() * sizeof(int), cudaMemcpyHostToDevice, p.stream));
    w.usable = true;
}

static size_t wide_smem_bytes(int nbins, int maxloc) {
    return 1024 + 4 * (size_t)kWideN * 128 + 2 * (size_t)nbins * kStageLd * 4 + (size_t)maxloc * 8 + 16 +
           (size_t)kWideN * sizeof(WideRight);
}

static bool launch_wide(Plan &p, const float *islab, long long npts, long long slab_stride, bool quads) {
    // The narrow orientation measured faster on the headline workload (shared
    // memory and tensor-memory contention slow the wide N = 256 MMAs to about
    // twice their isolated cost, and each right-row group re-reads the shell
    // fields); the wide kernel is selected per plan with FBS_OPT_TC_WIDE.
    if (!p.tc_wide) return false;
    TcState &st = tc_state(p);
    WideJob &w = quads ? st.wquad : st.wtrip;
    if (!w.built) build_wide(p, quads, w);
    if (!w.usable || wide_smem_bytes(p.nbins, w.maxloc) > 225 * 1024) return false;
    const int ngrp = (w.nright + kWideN - 1) / kWideN;
    int sms = 0, dev = 0;
    FBS_CUDA(cudaGetDevice(&dev));
    FBS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int G = std::max(1, sms / ngrp);
    if (G > p.part_blocks) G = p.part_blocks;
    const size_t sm = std::max<size_t>(wide_smem_bytes(p.nbins, w.maxloc), 116 * 1024);
    const TaskList &t = quads ? p.qtask : p.ttask;
    KTimer tm(p, quads ? KC_QUAD_TC : KC_CONTRACT_TC);
    FBS_CUDA(cudaFuncSetAttribute(contract_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid(G, ngrp);
    contract_wide_kernel<<<grid, kWideThreads, sm, p.stream>>>(
        islab, slab_stride, npts, p.nbins, w.nleft, w.d_left, w.d_rights, w.nright, w.d_item_out, t.nitems,
        quads ? p.d_qpart : p.d_tpart, p.precision == FBS_PREC_BF16 ? 0 : 1, 16, st.d_err, tc_wait_limit(p));
    FBS_CUDA(cudaGetLastError());
    return true;
}

// Shape of a level's tensor-core job (which: 0 triplets, 1 quadruplets, 2
// fused): built, usable, outer tiles (largest CTA group), inner rows, Npad,
// and of its latest launch the merged flag and points per step / 64.
void tc_job_info(Plan &p, int which, int32_t *out) {
    for (int i = 0; i < 11; ++i) out[i] = 0;
    if (!p.tc) return;
    TcState &st = *reinterpret_cast<TcState *>(p.tc);
    const TcJob &j = which == 0 ? st.trip : which == 1 ? st.quad : st.fused;
    out[0] = j.built;
    out[1] = j.usable;
    out[2] = j.maxtiles;
    out[3] = j.ninner;
    out[4] = j.Npad;
    out[5] = j.last_merged;
    out[6] = j.last_ka;
    out[7] = j.last_nst;
    out[8] = j.last_nsb;
    out[9] = j.last_nstg;
    out[10] = j.last_bfa;
}

int *tc_error_flag(Plan &p) { return p.root().d_errbuf; }
int *tc_sticky_flag(Plan &p) { return p.root().d_errbuf ? p.root().d_errbuf + 1 : nullptr; }

bool tc_quads_usable(Plan &p) {
    TcState &st = tc_state(p);
    if (!st.wquad.built) build_wide(p, true, st.wquad);
    if (st.wquad.usable) return true;
    if (!st.quad.built) build_job(p, p.qtask, true, st.quad);
    return st.quad.usable;
}

// cuTensorMapEncodeTiled through cudaGetDriverEntryPointByVersion, so the
// library links only the CUDA runtime (not libcuda directly).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// Tensor map of one slab of shell fields: x = point (npts valid, contiguous),
// y = bin (stride slab_stride floats); boxes of 32 points x all bins in the
// 128-byte swizzle; points past npts read as zero.
static CUtensorMap field_tensor_map(const float *islab, long long npts, long long slab_stride, int nbins,
                                    int rows) {
    auto enc = tensor_map_encoder();
    if (!enc) throw Failure{FBS_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
    if ((reinterpret_cast<uintptr_t>(islab) & 15) || ((slab_stride * 4) & 15) || nbins < 1 || nbins > 256 ||
        rows < nbins || npts < 1 || npts >= (1LL << 31))
        throw Failure{FBS_ERR_ARG, "shell-field slab does not meet the TMA layout rules"};
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)npts, (cuuint64_t)rows};  // rows: nbins per field of a batch
    cuuint64_t strides[1] = {(cuuint64_t)slab_stride * 4};
    cuuint32_t box[2] = {32u, (cuuint32_t)nbins};
    cuuint32_t es[2] = {1u, 1u};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(islab), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Failure{FBS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
    return m;
}

static void launch_job(Plan &p, TcJob &job, const float *islab, long long npts, long long slab_stride,
                       double *part, int nitems_total, int kclass, int nf) {
    TcState &st = tc_state(p);
    const int ngrp = (int)job.grp.size() - 1;
    int sms = 0, dev = 0;
    FBS_CUDA(cudaGetDevice(&dev));
    FBS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // CTAs per field and tile group: one wave of one CTA per SM over all of them
    int G = std::max(1, sms / (ngrp * nf));
    if (G > p.part_blocks) G = p.part_blocks;
    // 16 warps form the pair products and build operand B in turn (measured
    // faster at both headline passes); 8 + 8 concurrent roles on request
    const int aw = p.tc_roles == 2 ? 8 : 16;
    // 128-point chunks (half the hand-offs per point) when two 128-column A
    // stages fit beside the accumulators in tensor memory and shared memory
    // holds the doubled stages; 64-point chunks otherwise
    // BF16x3 with the hi and lo rows of B in one MMA (N = 2 Npad; two MMAs per
    // k-step instead of three) when the doubled accumulators still leave room
    // for two 128-column A stages in tensor memory
    const int x3 = p.precision == FBS_PREC_BF16 ? 0 : 1;
    int tstr = tile_stride(job.Npad);
    int acc_cols_max = (((job.maxtiles * tstr) + 31) / 32) * 32;
    const bool fits2 = acc_cols_max + 2 * 2 * kAStageCols <= 512 &&
                       tc_smem_bytes(p.nbins, job.Npad, job.maxloc, job.maxtiles, 2, 2) <= 220 * 1024;
    const int ka = (fits2 && p.tc_chunk != 1 && aw == 16) ? 2 : 1;
    int merged = 0;
    if (x3 && p.tc_merge != 1 && 2 * job.Npad <= 256) {
        const int acc2 = (((job.maxtiles * tile_stride(2 * job.Npad)) + 31) / 32) * 32;
        if (acc2 + 2 * ka * kAStageCols <= 512) {
            merged = 1;
            tstr = tile_stride(2 * job.Npad);
            acc_cols_max = acc2;
        }
    }
    // inner pair rows from operand A: one pair tile (so one CTA group), 16
    // producer warps, 128-point steps
    const int *ifeed = (job.d_ifeed && p.tc_bfroma == 0 && aw == 16 && ka == 2 && ngrp == 1) ? job.d_ifeed : nullptr;
    // A's hi and lo stacked on M (one MMA per k-step, the lo*lo products too):
    // one tile of at most 64 pairs with merged B, 16 producer warps, no feed;
    // its second set of compensated sums doubles the item sums in shared memory
    int stacked = (merged && !ifeed && p.tc_stack == 0 && aw == 16 && job.ntiles == 1 && ngrp == 1 &&
                   job.npairs <= 64) ? 1 : 0;
    if (stacked && tc_smem_bytes(p.nbins, job.Npad, 2 * job.maxloc, job.maxtiles, 2, ka, 2) > 220 * 1024) stacked = 0;
    const int sums = (stacked ? 2 : 1) * job.maxloc;
    // pipeline depths: 3 A stages when tensor memory allows; operand-B and
    // field stages as shared memory allows, the first of (B, field) = (4, 4),
    // (3, 4), (2, 4), (3, 2), (2, 2) that fits (FBS_OPT_TC_BSTAGES asks for a
    // B depth; with many bins four field stages measured faster than a third
    // B stage)
    const int nst = acc_cols_max + 3 * ka * kAStageCols <= 512 ? 3 : 2;
    const int want_nsb = p.tc_bstages;
    const auto fits = [&](int b, int f) {
        return tc_smem_bytes(p.nbins, job.Npad, sums, job.maxtiles, f, ka, b) <= 220 * 1024;
    };
    static const int order[5][2] = {{4, 4}, {3, 4}, {2, 4}, {3, 2}, {2, 2}};
    int nsb = 2, nstg = 2;  // fits: the job's tables (and the stacked sums) were sized for it
    const auto pick = [&](int want) {
        for (const auto &o : order)
            if ((!want || o[0] == want) && fits(o[0], o[1])) {
                nsb = o[0];
                nstg = o[1];
                return true;
            }
        return false;
    };
    if (!pick(want_nsb)) pick(0);
    const size_t sm = tc_smem_bytes(p.nbins, job.Npad, sums, job.maxtiles, nstg, ka, nsb);
    const int flush_every = 16 / ka;  // 1024 points in FP32 per flush
    const CUtensorMap fmap = field_tensor_map(islab, npts, slab_stride, p.nbins, nf * p.nbins);
    KTimer tm(p, kclass);
    dim3 grid(G, ngrp, nf);
    job.last_merged = stacked ? 2 : merged;
    job.last_ka = ka;
    job.last_nsb = nsb;
    job.last_nstg = nstg;
    job.last_nst = nst;
    const int nbuild = ifeed ? job.nsingle : job.ninner;
    job.last_bfa = ifeed ? job.ninner - job.nsingle : 0;
#define FBS_TC_LAUNCH(A, S, W, K, F)                                                                  \
    if (nst == A && nstg == S && aw == W && ka == K && (ifeed != nullptr) == F) {                   \
        launched = true;                                                                              \
        FBS_CUDA(cudaFuncSetAttribute(contract_tc_kernel<A, S, W, K, F>,                                 \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));          \
        contract_tc_kernel<A, S, W, K, F><<<grid, kTcThreads, sm, p.stream>>>(                          \
            fmap, npts, p.nbins, job.Npad, tstr, job.ninner, job.d_inner, job.d_pairs, job.npairs,      \
            job.d_grp, job.d_iout, nitems_total, part, x3, flush_every, st.d_err, tc_wait_limit(p),     \
            p.part_blocks, merged, nsb, ifeed, nbuild, stacked);                                      \
    }
    bool launched = false;
    FBS_TC_LAUNCH(2, 2, 16, 1, false)
    FBS_TC_LAUNCH(2, 4, 16, 1, false)
    FBS_TC_LAUNCH(3, 2, 16, 1, false)
    FBS_TC_LAUNCH(3, 4, 16, 1, false)
    FBS_TC_LAUNCH(2, 2, 8, 1, false)
    FBS_TC_LAUNCH(2, 4, 8, 1, false)
    FBS_TC_LAUNCH(3, 2, 8, 1, false)
    FBS_TC_LAUNCH(3, 4, 8, 1, false)
    FBS_TC_LAUNCH(2, 2, 16, 2, false)
    FBS_TC_LAUNCH(2, 2, 16, 2, true)
    FBS_TC_LAUNCH(2, 4, 16, 2, false)
    FBS_TC_LAUNCH(2, 4, 16, 2, true)
    FBS_TC_LAUNCH(3, 2, 16, 2, false)
    FBS_TC_LAUNCH(3, 2, 16, 2, true)
    FBS_TC_LAUNCH(3, 4, 16, 2, false)
    FBS_TC_LAUNCH(3, 4, 16, 2, true)
#undef FBS_TC_LAUNCH
    if (!launched) throw Failure{FBS_ERR_STATE, "tensor-core contraction: no kernel for this pipeline shape"};
    FBS_CUDA(cudaGetLastError());
}

void launch_contract_tc(Plan &p, const float *islab, long long npts, long long slab_stride, bool quads,
                        int nf, double *part) {
    const TaskList &t = quads ? p.qtask : p.ttask;
    if (t.nitems == 0) return;
    if (nf == 1 && launch_wide(p, islab, npts, slab_stride, quads)) return;  // batches: narrow only
    TcState &st = tc_state(p);
    TcJob &job = quads ? st.quad : st.trip;
    if (job.built && !quads && job.variant != p.tc_pairs) job = TcJob{};  // option changed: rebuild
    if (!job.built) build_job(p, t, quads, job);
    if (!job.usable)
        throw Failure{FBS_ERR_ARG, "tensor-core contraction: more than 256 inner rows or shared memory exceeded"};
    launch_job(p, job, islab, npts, slab_stride, part ? part : (quads ? p.d_qpart : p.d_tpart), t.nitems,
               quads ? KC_QUAD_TC : KC_CONTRACT_TC, nf);
}

bool tc_fused_usable(Plan &p) {
    if (p.tc_wide || p.ttask.nitems == 0 || p.qtask.nitems == 0) return false;
    TcState &st = tc_state(p);
    if (st.fused.built && st.fused.variant != p.tc_pairs) st.fused = TcJob{};  // option changed: rebuild
    if (!st.fused.built) build_fused_job(p, st.fused);
    return st.fused.usable;
}

void launch_contract_tc_fused(Plan &p, const float *islab, long long npts, long long slab_stride) {
    TcState &st = tc_state(p);
    launch_job(p, st.fused, islab, npts, slab_stride, p.d_fpart, p.ttask.nitems + p.qtask.nitems,
               KC_QUAD_TC, 1);
}

void free_tc_state(Plan &p) {
    if (!p.tc) return;
    delete reinterpret_cast<TcState *>(p.tc);  // device buffers belong to the plan's allocation list
    p.tc = nullptr;
}

}  // namespace fbs
