// Split-BF16 tensor-core (tcgen05 / TMEM) kernels for sm_103a.
//
// k_tc (phase modes): the phase contraction of eq. Emat,
// Phi = (2 theta . P_A) S_Z^T, one 128 (observables) x 256 (samples) FP32
// accumulator in TMEM per CTA and tile, K = gates streamed in 64-wide stages.
// Operands never exist in HBM as numbers: a TMA warp brings 256-gate slices
// of the parity bits (and of the hi/lo BF16 split of 2 theta) into shared
// memory, and sixteen producer warps expand them: B = 1 - 2 P_Z into the
// 128-byte-swizzled K-major BF16 layout in shared memory, and A_hi =
// hi_j [P_A], A_lo = lo_j [P_A] (all exact in BF16) either straight into
// TMEM with tcgen05.st (the default for CTA pairs: the MMA then reads A from
// TMEM, and shared memory carries only B) or into shared memory like B
// (IQP_PHASE_TMEM=0, and the one-CTA form). One thread issues two
// tcgen05.mma per 16-gate step (hi and lo share B), a whole stage from one
// asm statement. The epilogue runs in the producer warps straight from TMEM:
//   mode 0: cos, per-observable (S, M2) partials over 64-sample groups, and
//           Phi itself (FP32) when a gradient pass follows that reads it back
//           (the MMD loss, the autograd pair; k_w_from_phi forms W from it);
//   mode 1: W = sin Phi (alpha + beta cos Phi), split into hi + lo BF16 rows;
//   mode 2: both from one pass (the loss coefficients known in advance).
// Otherwise Phi itself is never written.
//
// Two sample tiles per tile (TA = 3; the full rounds of tiles of CTA
// pairs): a pair computes 256 observables x 512 samples against each A stage,
// in two M256 x N256 accumulators that fill TMEM (columns 0..255, 256..511).
// A_hi / A_lo then live in shared memory beside the two B operands, a stage
// takes sixteen MMAs, and the A expansion per flop halves. The running sums
// of the accumulation chunks go to a per-CTA buffer in global memory (it
// stays in L2). The double tiles of a last, partial round run as a balanced
// split (TcArgs::sk): their bits stages, end to end, in one equal range per
// CTA pair, each range's piece of a tile a split part; or, without room for
// its scratch, as single tiles (TcArgs::dtmap), split along the gates as
// below.
//
// Dense form (mode 3, A by TMA): out = (A_hi + A_lo) (1 - 2 B_bits)^T for a
// dense split-BF16 matrix A brought in by TMA and a +-1 operand expanded from
// bits as above, the FP32 accumulator stored as is (FP32 or FP64). The
// low-order form's pair contractions M = C S and H = (s o V) S^T use it.
//
// Gradient contraction (Sec. 2.4, backward of eq. Emat), two kernels:
//  - k_grad_pair (default): CTA pairs in the transposed orientation,
//    D[j][a] = sum_i S_Z[i][j] W[a][i] over 256 gates x 256 observables per
//    tile, K = samples in 128-wide stages, the +-1 operand written into TMEM
//    from P_Z^T bits, W_hi / W_lo by TMA; the epilogue masks by 2 P_A[a][j]
//    (bits of P_A^T) and sums over the tile's observables per gate row
//    (description at the kernel);
//  - k_tc<GRAD> (IQP_GRAD_PAIR=0): one CTA per 128 observables x 256 gates,
//    W tiles by TMA as A, the +-1 operand expanded into shared memory from
//    P_Z^T, reduced over observables with a warp reduce-scatter.
// Both write FP64 partials per (observable tile, gate) that k_grad_reduce
// sums in a fixed order.
//
// Accumulation: the tensor core's FP32 accumulation rounds toward zero, so a
// single accumulator over ~10^4 K-steps shrinks |Phi| by ~1e-4 relative. Each
// tile therefore accumulates in chunks of `chunk` K-stages: a chunk starts a
// fresh accumulator (TMEM columns 0..255) and, when it completes, the
// producer warps add it into an FP32 running sum with round-to-nearest adds
// (TMEM columns 256..511, or shared memory when A occupies those columns, or
// global memory in the two-sample-tile form).
// The epilogue reads accumulator + running sum. The pair gradient reduces
// every chunk into its FP64 per-gate partials instead.
//
// CTA pairs: with CG = 2 the kernels run as clusters of two CTAs on two SMs.
// A phase tile is 256 observables x 256 samples; each CTA holds 128
// observables' A rows and half (128 rows) of the B operand, and the even CTA
// issues M256 x N256 pair MMAs (cta_group::2) that read both CTAs' operands
// and write 128 accumulator rows into each CTA's TMEM. Per SM this halves the
// B operand's expansion work and the tensor core's B reads. Both CTAs'
// producer warps arrive on the even CTA's stage barrier (the odd CTA's through
// one forwarding thread); stage and chunk completions are signalled to both
// CTAs by one pair commit.
//
// Every wait is bounded (globaltimer); on expiry the CTA records
// IQP_ERR_TIMEOUT, drains its in-flight copies and MMAs, frees TMEM and exits.
#include <cuda.h>

#include <cstdlib>

#include "common.cuh"

namespace iqp {

uint64_t default_spin_limit_ns();
uint32_t check_word_tc() { return take_check_word(); }

namespace {

constexpr int TM = 128;      // accumulator rows (observables) per CTA
constexpr int TN = 256;      // accumulator columns (samples or gates) per tile
constexpr int KS = 64;       // K per operand stage
constexpr int KB = 256;      // K per bits stage
constexpr int NBITS = 2;     // bits stages
constexpr int NGEN = 16;     // producer / epilogue warps (4 per scheduler)
constexpr int kThreads = 64 + NGEN * 32;
constexpr int kRowsPerPass = NGEN * 32 / 8;   // operand rows expanded per pass (8 chunks per row)
constexpr int kGroupCols = TN / (NGEN / 4);   // accumulator columns per epilogue warp
constexpr int kGroupLoads = kGroupCols / 32;
constexpr uint32_t kTmemCols = 512;   // accumulator (0..255) + running sum (256..511)
constexpr uint32_t kSumCol = 256;
// A-in-TMEM form: columns 256..511 hold the A operand of the four operand
// stages instead of the running sum: stage os at 256 + 64 os; its 16-gate
// K step k (0..3) has A_hi at + 16 k and A_lo at + 16 k + 8 (8 columns of
// two BF16 each), so one warp's share is 16 contiguous columns.
constexpr uint32_t kAColBase = 256;
constexpr uint32_t kAColStage = 64;
constexpr int kMaxOp = 4;
constexpr int kWPrefetch = 8;  // gradient: W tiles prefetched into L2 this many stages ahead

// Shared-memory layout for a CTA group of CG CTAs (CG = 1 or 2). ATM: the A
// operand (hi / lo) lives in TMEM, so an operand stage in shared memory holds
// only B, and the running sum of the accumulation chunks moves from TMEM to
// shared memory (TM x TN FP32, as float4 groups of 4 columns, row-minor).
// DT (two sample tiles per tile): an operand stage holds A_hi, A_lo and the
// B operands of both sample tiles, the two accumulators fill TMEM, and the
// running sums live in global memory.
template <int CG, bool ATMA, bool ATM = false, bool DT = false>
struct Cfg {
    static constexpr int TNB = TN / CG;      // B rows this CTA holds (per sample tile)
    static constexpr int NOP = DT ? 3 : (CG == 2 || ATM) ? 4 : (ATMA ? 3 : 2);  // operand stages
    // Operand stage: A_hi (128 x 128 B), A_lo, B (TNB x 128 B) [DT: then the
    // second sample tile's B]; ATM: B only.
    static constexpr uint32_t OP_A_HI = 0, OP_A_LO = 16384, OP_B = ATM ? 0 : 32768;
    static constexpr uint32_t OP_B1 = OP_B + TNB * 128;
    static constexpr uint32_t OP_BYTES = ATM ? TNB * 128 : 32768 + (DT ? 2 : 1) * TNB * 128;
    // Bits stage: A bits (128 rows x 32 B), B bits (TNB rows x 32 B) [DT: then
    // the second sample tile's], c_hi, c_lo.
    static constexpr uint32_t BT_A = 0, BT_B = 4096, BT_B1 = BT_B + TNB * 32;
    static constexpr uint32_t BT_CHI = BT_B + (DT ? 2 : 1) * TNB * 32, BT_CLO = BT_CHI + 512;
    static constexpr uint32_t BT_BYTES = BT_CLO + 512;
    static constexpr uint32_t SM_OP = 0;
    static constexpr uint32_t SM_BITS = SM_OP + NOP * OP_BYTES;
    static constexpr uint32_t SM_BAR = SM_BITS + NBITS * BT_BYTES;
    static constexpr uint32_t SM_RED = SM_BAR + 256;   // 4 x 256 floats (grad epilogue)
    static constexpr uint32_t SM_SUM = SM_RED + 4 * 256 * 4;  // ATM: running sum
    static constexpr uint32_t SM_END = SM_SUM + (ATM ? TM * TN * 4 : 0);
    static constexpr uint32_t SMEM = SM_END + 1024;     // + alignment slack
    static constexpr uint32_t IDESC = idesc_bf16(TM * CG, TN);
    static_assert(OP_BYTES % 1024 == 0 && BT_BYTES % 1024 == 0 && SM_SUM % 16 == 0, "stage alignment");
    static_assert(SMEM <= 232448, "shared memory");
};

// Tile t -> (row block tm, column block tc), walking `gm` row blocks of one
// column block before the next column block (the last group may be
// shorter). The CTAs running at once then share gm row panels and about
// (CTAs / gm) column panels, which stay in L2: each column panel is read
// from DRAM once per group instead of once per row block.
__device__ __forceinline__ void tile_coords(int64_t t, int64_t tiles_m, int64_t tiles_nc, int64_t gm, int64_t &tm,
                                            int64_t &tc) {
    const int64_t per = gm * tiles_nc;
    const int64_t g = t / per;
    const int64_t r = t - g * per;
    const int64_t rows = tiles_m - g * gm < gm ? tiles_m - g * gm : gm;
    tm = g * gm + r % rows;
    tc = r / rows;
}

struct TcArgs;
__device__ __forceinline__ void tile_rc(int64_t t, const TcArgs &a, int64_t &tm, int64_t &tc);

struct TcArgs {
    int64_t l, s, m;
    int64_t nks;          // operand stages per tile
    int64_t chunk;        // operand stages per accumulation chunk
    int64_t tiles_m, tiles_n;
    int64_t group_m;      // row blocks per tile group (L2 rasterisation)
    const __nv_bfloat16 *chi, *clo;
    int64_t mpad;          // length of chi / clo
    double2 *part;
    int64_t nparts;
    const double *alpha, *beta;
    __nv_bfloat16 *whi, *wlo;
    int64_t ldw;
    const uint32_t *pa32;  // P_A, for the gradient mask
    int64_t ldp32;
    double *gpart;
    void *out;             // mode 3: the accumulator stored as is (FP32, or FP64 if out_f64)
    int64_t ldo;
    int out_f64;
    // Work units of this launch: the tiles, whole (nunits tiles); or, for a
    // split launch, nunits parts of the tiles from `whole` on, nsplit parts
    // per tile (phase modes only).
    int64_t nunits, whole;
    int nsplit;
    float *skp;            // split parts' partial accumulators, TM x TN FP32 per (part, CTA of the pair)
    int *skc;              // per (split tile, CTA of the pair): parts finished so far
    uint32_t *status;
    uint64_t limit_ns;
    int serp;              // phase, whole tiles: every other round of tiles walks the gates backwards
    // Two-sample-tile phase kernels: per CTA, the running sums of both
    // accumulators (2 x TM x TN FP32 as float4 groups of 4 columns, row-minor).
    float4 *gsum;
    // Single tiles taken from double tiles (the last round of a two-tile
    // phase): tile t is half t % 2 of double tile dbase + t / 2 of a
    // tiles_m x tiles_n2 walk.
    int dtmap;
    int64_t dbase, tiles_n2;
    // Balanced split of a last round (sk = 1; split units only): the skW
    // bits stages of the tiles from `whole` on, laid end to end, are cut into
    // skP equal contiguous ranges, one per CTA group; unit u is piece u / skP
    // of range u % skP (the part of the range inside one tile; empty when the
    // range has fewer pieces). The pieces of tile whole + t take the slots
    // t * skKP + j, j = 0, 1, ... in range order.
    int sk;
    int64_t skW, skP, skKP;
    int64_t skcap;  // floats of split-part scratch at skp
};

__device__ __forceinline__ void tile_rc(int64_t t, const TcArgs &a, int64_t &tm, int64_t &tc) {
    if (a.dtmap) {
        int64_t tc2;
        tile_coords(a.dbase + t / 2, a.tiles_m, a.tiles_n2, a.group_m, tm, tc2);
        tc = 2 * tc2 + (t & 1);
        return;
    }
    tile_coords(t, a.tiles_m, a.tiles_n, a.group_m, tm, tc);
}

struct Bars {
    uint64_t bits_full[NBITS], bits_empty[NBITS], op_full[kMaxOp], op_empty[kMaxOp], w_full[kMaxOp],
        peer_full[kMaxOp], acc_full, drain, red_full, part_done, part_flag;
    uint32_t tmem_slot;
    int abort_flag;
    int last_flag;  // this CTA finished the last part of a split tile
};

// Work unit u -> its tile, its operand-stage range [ks0, ks1) and, for a
// part of a split tile, its slot v (-1 for a whole tile). SPL = false: the
// units are the tiles, whole. SPL = true: unit u is part u % nsplit of tile
// whole + u / nsplit; the parts cover the tile's stages in ranges of whole
// bits stages (KB / KS operand stages), in order.
template <bool SPL>
__device__ __forceinline__ void unit_of(int64_t u, const TcArgs &a, int nks, int64_t &tile, int &ks0, int &ks1,
                                        int64_t &v) {
    if (!SPL) {
        tile = u;
        ks0 = 0;
        ks1 = nks;
        v = -1;
        return;
    }
    const int64_t nkb = (nks + KB / KS - 1) / (KB / KS);
    if (a.sk) {
        const int64_t g = u % a.skP, k = u / a.skP;
        const int64_t A = g * a.skW / a.skP, B = (g + 1) * a.skW / a.skP;
        const int64_t start = k == 0 ? A : (A / nkb + k) * nkb;
        tile = a.whole;
        ks0 = ks1 = 0;
        v = -1;
        if (start >= B) return;  // this range has no piece k
        const int64_t t = start / nkb;
        const int64_t end = B < (t + 1) * nkb ? B : (t + 1) * nkb;
        tile = a.whole + t;
        ks0 = (KB / KS) * (int)(start - t * nkb);
        const int64_t e = (KB / KS) * (end - t * nkb);
        ks1 = e < nks ? (int)e : nks;
        // the range holding the tile's first bits stage: the largest g0 with g0 W / P <= t nkb
        const int64_t g0 = ((t * nkb + 1) * a.skP - 1) / a.skW;
        v = t * a.skKP + (g - g0);
        return;
    }
    v = u;
    tile = a.whole + v / a.nsplit;
    const int64_t part = v % a.nsplit;
    ks0 = (KB / KS) * (int)(part * nkb / a.nsplit);
    const int e = (KB / KS) * (int)((part + 1) * nkb / a.nsplit);
    ks1 = e < nks ? e : nks;
}

// A split unit's slot v -> its tile's index tt among the split tiles, the
// number of parts of that tile and the slot of its first part.
__device__ __forceinline__ void part_info(int64_t v, const TcArgs &a, int nks, int64_t &tt, int64_t &np,
                                          int64_t &base) {
    if (a.sk) {
        const int64_t nkb = (nks + KB / KS - 1) / (KB / KS);
        tt = v / a.skKP;
        const int64_t g0 = ((tt * nkb + 1) * a.skP - 1) / a.skW;
        const int64_t g1 = ((tt + 1) * nkb * a.skP - 1) / a.skW;
        np = g1 - g0 + 1;
        base = tt * a.skKP;
        return;
    }
    tt = v / a.nsplit;
    np = a.nsplit;
    base = tt * a.nsplit;
}

__device__ __forceinline__ uint8_t *aligned_smem(uint8_t *raw) {
    const uint32_t a = smem_u32(raw);
    return raw + ((1024u - (a & 1023u)) & 1023u);
}

// Expand one 64-gate sub-stage q of a bits stage into the B operand
// (ROWS rows, +-1 BF16). Thread gt handles chunk gt%8 of rows
// gt/8 + kRowsPerPass*k.
template <int ROWS>
__device__ __forceinline__ void expand_b(const uint8_t *bits, uint8_t *opB, int q, int gt) {
    const uint32_t c = gt & 7;
    const uint32_t sub = (uint32_t)q * 8u + (c >> 2) * 4u;  // byte offset of the u32 holding chunk c
    const uint32_t sh = (c & 3u) * 8u;
#pragma unroll
    for (int k = 0; k < ROWS / kRowsPerPass; ++k) {
        const uint32_t row = (uint32_t)(gt >> 3) + (uint32_t)kRowsPerPass * k;
        const uint32_t w = *reinterpret_cast<const uint32_t *>(bits + row * 32u + sub);
        const uint4 v = expand_pm1((w >> sh) & 0xFFu);
        *reinterpret_cast<uint4 *>(opB + swz128(row, c)) = v;
    }
}

// Expand sub-stage q into A_hi / A_lo (128 rows): hi_j / lo_j where the
// parity bit is set, 0 elsewhere.
__device__ __forceinline__ void expand_a(const uint8_t *bitsA, const uint8_t *chi, const uint8_t *clo, uint8_t *opHi,
                                         uint8_t *opLo, int q, int gt) {
    const uint32_t c = gt & 7;
    const uint4 h = *reinterpret_cast<const uint4 *>(chi + (uint32_t)q * 128u + c * 16u);
    const uint4 lo = *reinterpret_cast<const uint4 *>(clo + (uint32_t)q * 128u + c * 16u);
    const uint32_t sub = (uint32_t)q * 8u + (c >> 2) * 4u;
    const uint32_t sh = (c & 3u) * 8u;
#pragma unroll
    for (int k = 0; k < TM / kRowsPerPass; ++k) {
        const uint32_t row = (uint32_t)(gt >> 3) + (uint32_t)kRowsPerPass * k;
        const uint32_t w = *reinterpret_cast<const uint32_t *>(bitsA + row * 32u + sub);
        const uint4 mk = expand_mask((w >> sh) & 0xFFu);
        const uint32_t off = swz128(row, c);
        *reinterpret_cast<uint4 *>(opHi + off) = make_uint4(h.x & mk.x, h.y & mk.y, h.z & mk.z, h.w & mk.w);
        *reinterpret_cast<uint4 *>(opLo + off) = make_uint4(lo.x & mk.x, lo.y & mk.y, lo.z & mk.z, lo.w & mk.w);
    }
}

// Sum over the 32 lanes of v[lane][k]: afterwards lane L returns the sum of column L.
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = upper ? v[k] : v[k + w];
            const float keep = upper ? v[k + w] : v[k];
            v[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, w);
        }
    }
    return v[0];
}

// Bounded wait polled by every lane (each needs the acquire), with the outcome
// made warp-uniform so that a give-up never splits a warp.
__device__ __forceinline__ bool wait_warp(uint64_t *b, uint32_t parity, volatile int *abort_flag, uint32_t *status,
                                          uint64_t lim) {
    const bool got = mbar_wait(b, parity, abort_flag, status, lim);
    return __all_sync(0xFFFFFFFFu, got);
}

// wait_warp with cluster-scope acquire (the barrier completes from the peer CTA too).
__device__ __forceinline__ bool wait_warp_cluster(uint64_t *b, uint32_t parity, volatile int *abort_flag,
                                                  uint32_t *status, uint64_t lim) {
    const bool got = mbar_wait_cluster(b, parity, abort_flag, status, lim);
    return __all_sync(0xFFFFFFFFu, got);
}

// 32 columns of the tile at TMEM address `t`: the current accumulator plus,
// when the tile was accumulated in more than one chunk, the running sum (in
// TMEM at t + kSumCol, or, when `ss` is given, in shared memory: the 8 float4
// groups of these columns for this thread's row at ss[0], ss[TM], ...).
__device__ __forceinline__ void load_sum32(uint32_t t, bool chunked, uint32_t (&r)[32], const float4 *ss = nullptr) {
    tmem_ld32(t, r);
    if (chunked) {
        if (ss != nullptr) {
#pragma unroll
            for (int e4 = 0; e4 < 8; ++e4) {
                const float4 v = ss[e4 * TM];
                r[4 * e4] = __float_as_uint(__uint_as_float(r[4 * e4]) + v.x);
                r[4 * e4 + 1] = __float_as_uint(__uint_as_float(r[4 * e4 + 1]) + v.y);
                r[4 * e4 + 2] = __float_as_uint(__uint_as_float(r[4 * e4 + 2]) + v.z);
                r[4 * e4 + 3] = __float_as_uint(__uint_as_float(r[4 * e4 + 3]) + v.w);
            }
            return;
        }
        uint32_t acc[32];
        tmem_ld32(t + kSumCol, acc);
#pragma unroll
        for (int e = 0; e < 32; ++e) r[e] = __float_as_uint(__uint_as_float(r[e]) + __uint_as_float(acc[e]));
    }
}

// A-in-TMEM form: this warp's share of one 64-gate operand stage of A, the 16
// gates [16 g, 16 g + 16) (K step g) for the row of TMEM lane
// (32 quarter + lane): hi_j (A_hi) and lo_j (A_lo) where bit j of `b16` (the
// row's parities of these gates) is set, 0 elsewhere, two BF16 per 32-bit
// column (the lower gate in the low half). chi / clo: the bits stage's hi /
// lo split of 2 theta; q: the operand stage within the bits stage. `t` is the
// TMEM address of the warp's 16 columns: A_hi in the first 8, A_lo in the
// next 8, stored at once.
__device__ __forceinline__ void expand_a_tmem(uint32_t b16, const uint8_t *chi, const uint8_t *clo, int q, int g,
                                              uint32_t t) {
    const uint32_t off = (uint32_t)q * 128u + (uint32_t)g * 32u;
    const uint4 h0 = *reinterpret_cast<const uint4 *>(chi + off);
    const uint4 h1 = *reinterpret_cast<const uint4 *>(chi + off + 16);
    const uint4 l0 = *reinterpret_cast<const uint4 *>(clo + off);
    const uint4 l1 = *reinterpret_cast<const uint4 *>(clo + off + 16);
    const uint4 m0 = expand_mask(b16 & 0xFFu), m1 = expand_mask((b16 >> 8) & 0xFFu);
    const uint32_t v[16] = {h0.x & m0.x, h0.y & m0.y, h0.z & m0.z, h0.w & m0.w,
                            h1.x & m1.x, h1.y & m1.y, h1.z & m1.z, h1.w & m1.w,
                            l0.x & m0.x, l0.y & m0.y, l0.z & m0.z, l0.w & m0.w,
                            l1.x & m1.x, l1.y & m1.y, l1.z & m1.z, l1.w & m1.w};
    tmem_st16(t, v);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
    const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
    return lo | (hi << 16);
}

// W = sin Phi (alpha_a + beta_a cos Phi) as BF16 hi/lo (l x ldw) from a Phi
// the statistics pass kept (l x ldphi FP32, columns < s), with the
// arithmetic of the recompute epilogue, so W is the same bit for bit. Four
// samples per thread; columns >= s get zeros (the gradient's tensor map ends
// at s).
__global__ void __launch_bounds__(256) k_w_from_phi(const float *__restrict__ phi, int64_t ldphi, int64_t ldw,
                                                    int64_t l, int64_t s,
                                                    const double *__restrict__ alpha,
                                                    const double *__restrict__ beta, __nv_bfloat16 *__restrict__ whi,
                                                    __nv_bfloat16 *__restrict__ wlo) {
    const int64_t per_row = ldw / 4;
    const int64_t total = l * per_row;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = g / per_row, i0 = (g - row * per_row) * 4;
        if (i0 >= s) continue;
        if (!IQP_IN(row, l, 40) || !IQP_IN(row * ldphi + i0 + 3, l * ldphi, 41) || !IQP_IN(row * ldw + i0 + 3, l * ldw, 42))
            continue;
        const float al = (float)alpha[row];
        const float be = beta ? (float)beta[row] : 0.f;
        const float4 f = *reinterpret_cast<const float4 *>(phi + row * ldphi + i0);
        const float v[4] = {f.x, f.y, f.z, f.w};
        uint32_t ph[2], pl[2];
#pragma unroll
        for (int e = 0; e < 4; e += 2) {
            float s0, k0, s1, k1;
            sincosf(v[e], &s0, &k0);
            sincosf(v[e + 1], &s1, &k1);
            const float w0 = i0 + e < s ? s0 * (al + be * k0) : 0.f;
            const float w1 = i0 + e + 1 < s ? s1 * (al + be * k1) : 0.f;
            const float h0 = __bfloat162float(__float2bfloat16_rn(w0));
            const float h1 = __bfloat162float(__float2bfloat16_rn(w1));
            ph[e / 2] = pack_bf16x2(h0, h1);
            pl[e / 2] = pack_bf16x2(w0 - h0, w1 - h1);
        }
        *reinterpret_cast<uint2 *>(whi + row * ldw + i0) = make_uint2(ph[0], ph[1]);
        *reinterpret_cast<uint2 *>(wlo + row * ldw + i0) = make_uint2(pl[0], pl[1]);
    }
}

// ------------------------------------------------------------------ kernel
// W hi/lo (BF16 pairs) of 32 consecutive samples i0.. of observable row.
__device__ __forceinline__ void store_w32(const TcArgs &args, int64_t row, int64_t i0, const uint32_t (&ph)[16],
                                          const uint32_t (&pl)[16]) {
    if (!IQP_IN(row * args.ldw + i0, args.l * args.ldw, 43) ||
        !IQP_IN(row * args.ldw + (i0 + 32 <= args.s ? i0 + 31 : args.s - 1), args.l * args.ldw, 44))
        return;
    __nv_bfloat16 *dh = args.whi + row * args.ldw + i0;
    __nv_bfloat16 *dl = args.wlo + row * args.ldw + i0;
    if (i0 + 32 <= args.s) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            reinterpret_cast<uint4 *>(dh)[v] = make_uint4(ph[4 * v], ph[4 * v + 1], ph[4 * v + 2], ph[4 * v + 3]);
            reinterpret_cast<uint4 *>(dl)[v] = make_uint4(pl[4 * v], pl[4 * v + 1], pl[4 * v + 2], pl[4 * v + 3]);
        }
    } else {
        uint16_t *sh = reinterpret_cast<uint16_t *>(dh);
        uint16_t *sl = reinterpret_cast<uint16_t *>(dl);
        for (int e = 0; e < 32 && i0 + e < args.s; ++e) {
            sh[e] = (uint16_t)(ph[e / 2] >> ((e & 1) * 16));
            sl[e] = (uint16_t)(pl[e / 2] >> ((e & 1) * 16));
        }
    }
}

// Accumulator values of 32 consecutive columns col0.. of `row`, stored into
// args.out (row-major, args.ldo elements per row, columns < args.s): FP32, or
// FP64 when args.out_f64. Rows start 16-byte aligned (ldo a multiple of 4).
__device__ __forceinline__ void store_out32(const TcArgs &args, int64_t row, int64_t col0, const uint32_t (&r)[32]) {
    if (!IQP_IN(row * args.ldo + col0, args.l * args.ldo, 45) ||
        !IQP_IN(row * args.ldo + (col0 + 32 <= args.s ? col0 + 31 : args.s - 1), args.l * args.ldo, 46))
        return;
    if (args.out_f64) {
        double *d = static_cast<double *>(args.out) + row * args.ldo + col0;
        if (col0 + 32 <= args.s) {
#pragma unroll
            for (int e = 0; e < 32; e += 2)
                *reinterpret_cast<double2 *>(d + e) =
                    make_double2((double)__uint_as_float(r[e]), (double)__uint_as_float(r[e + 1]));
        } else {
            for (int e = 0; e < 32 && col0 + e < args.s; ++e) d[e] = (double)__uint_as_float(r[e]);
        }
    } else {
        float *f = static_cast<float *>(args.out) + row * args.ldo + col0;
        if (col0 + 32 <= args.s) {
#pragma unroll
            for (int e = 0; e < 32; e += 4)
                *reinterpret_cast<float4 *>(f + e) = make_float4(__uint_as_float(r[e]), __uint_as_float(r[e + 1]),
                                                                 __uint_as_float(r[e + 2]), __uint_as_float(r[e + 3]));
        } else {
            for (int e = 0; e < 32 && col0 + e < args.s; ++e) f[e] = __uint_as_float(r[e]);
        }
    }
}

// Split phase tiles (kept out of line, so that their registers do not weigh
// on the stage loop). split_store: this warp's 32 rows x 64 columns of the
// accumulator (+ running sum) into its part's slot. split_sum: the sum of
// the tile's nsplit parts, in part order, into the accumulator columns.
__device__ __noinline__ void split_store(float *dst, uint32_t tbase, bool chunked, const float4 *ss0) {
    uint32_t r[32];
#pragma unroll 1
    for (int c = 0; c < kGroupLoads; ++c) {
        load_sum32(tbase + c * 32, chunked, r, ss0 != nullptr ? ss0 + c * 8 * TM : nullptr);
#pragma unroll
        for (int e = 0; e < 32; e += 4)
            *reinterpret_cast<float4 *>(dst + c * 32 + e) = make_float4(
                __uint_as_float(r[e]), __uint_as_float(r[e + 1]), __uint_as_float(r[e + 2]), __uint_as_float(r[e + 3]));
    }
}

__device__ __noinline__ void split_sum(const float *src0, int64_t part_stride, int nsplit, uint32_t tbase) {
#pragma unroll 1
    for (int c = 0; c < kGroupLoads; ++c) {
        uint32_t r[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) r[e] = 0u;  // +0.0f
        for (int pp = 0; pp < nsplit; ++pp) {
            const float *src = src0 + pp * part_stride + c * 32;
#pragma unroll
            for (int e = 0; e < 32; e += 4) {
                const float4 x = __ldcg(reinterpret_cast<const float4 *>(src + e));
                r[e] = __float_as_uint(__uint_as_float(r[e]) + x.x);
                r[e + 1] = __float_as_uint(__uint_as_float(r[e + 1]) + x.y);
                r[e + 2] = __float_as_uint(__uint_as_float(r[e + 2]) + x.z);
                r[e + 3] = __float_as_uint(__uint_as_float(r[e + 3]) + x.w);
            }
        }
        tmem_st32(tbase + c * 32, r);
    }
}

// GRAD = false: phase contraction (MODE 0 stats / MODE 1 W / MODE 2 both),
//              or (MODE 3) a dense contraction whose accumulator is stored.
// GRAD = true : gradient contraction.
// AT = true: the A operand arrives by TMA in the swizzled layout (always for
// the gradient's W; for MODE 3, a dense split-BF16 matrix); AT = false: the
// producer warps expand it from P_A bits and the hi/lo split of 2 theta.
// CG = 1: one CTA per tile of 128 rows; CG = 2: a CTA pair per tile of 256 rows.
// TA (phase modes of CTA pairs): 0 = A in shared memory; 1 = A in TMEM; 3 =
// two sample tiles (2 x 256 samples) per tile against each A stage.
template <bool GRAD, int MODE, int CG, bool AT, bool SPL, int TA>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
         const __grid_constant__ CUtensorMap tmB, const TcArgs args) {
    constexpr bool ATMA = GRAD || AT;  // A operand by TMA
    // A operand in TMEM, written by the producer warps (phase modes, CTA pairs)
    constexpr bool ATM = TA == 1 && !GRAD && !AT && CG == 2;
    // Two sample tiles per tile (phase modes, CTA pairs, whole tiles): A in
    // shared memory, two accumulators, running sums in global memory
    constexpr bool DT = TA == 3 && !GRAD && !AT && CG == 2;
    using C = Cfg<CG, ATMA, ATM, DT>;
    constexpr int NOP = C::NOP;
    // Serpentine gate order (phase kernels, whole tiles): the CTA groups' odd
    // rounds of tiles walk their bits stages from the last to the first, so a
    // round starts on the operand rows the round before it read last, which
    // are still in L2. The sum is the same up to the order of its terms.
    constexpr bool SERP = !GRAD && !ATMA && !SPL;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = aligned_smem(smem_raw);
    Bars *bar = reinterpret_cast<Bars *>(smem + C::SM_BAR);
    float *red = reinterpret_cast<float *>(smem + C::SM_RED);
    float4 *sum4 = reinterpret_cast<float4 *>(smem + C::SM_SUM);  // ATM: running sum
    volatile int *abort_flag = &bar->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = args.limit_ns;
    uint32_t *status = args.status;
    constexpr int CL = CG;  // CTAs per cluster
    const uint32_t crank = CL == 2 ? cluster_ctarank() : 0u;  // CTA rank in the cluster
    const bool leader = CG == 1 || crank == 0;                 // issues this CTA's MMAs
    const int64_t group0 = blockIdx.x / CL, ngroups = gridDim.x / CL;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NBITS; ++i) {
            mbar_init(&bar->bits_full[i], 1);
            mbar_init(&bar->bits_empty[i], NGEN);
        }
        for (int i = 0; i < NOP; ++i) {
            // Even CTA: its own producer warps, plus one forwarded arrival from
            // the odd CTA of a pair.
            mbar_init(&bar->op_full[i], CG == 2 ? NGEN + 1 : NGEN);
            mbar_init(&bar->op_empty[i], 1);  // the MMAs that read the stage
            mbar_init(&bar->w_full[i], 1);
            mbar_init(&bar->peer_full[i], NGEN);  // odd CTA: its producer warps
        }
        mbar_init(&bar->acc_full, 1);
        mbar_init(&bar->drain, 1);
        mbar_init(&bar->red_full, NGEN);
        mbar_init(&bar->part_done, NGEN);
        mbar_init(&bar->part_flag, 1);
        bar->last_flag = 0;
        bar->abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async_smem();
    }
    if (warp == 1) {
        if constexpr (CG == 2) {
            tmem_alloc_pair(&bar->tmem_slot, kTmemCols);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(&bar->tmem_slot, kTmemCols);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (CL == 2) cluster_sync_all();  // the peer's barriers exist before anyone arrives on them
    tc_fence_after();
    const uint32_t tmem = bar->tmem_slot;

    const int64_t nunits = args.nunits;
    const int nks = (int)args.nks;     // host guarantees nks < 2^31
    const int chunk = (int)args.chunk;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            prefetch_tmap(&tmA);
            prefetch_tmap(&tmB);
            if (ATMA) prefetch_tmap(&tmA2);
            uint32_t itb = 0, ito = 0;
            uint32_t bmask = 0, bpar = 0, omask = 0, opar = 0;  // issued stages and their last parities
            bool ok = true;
            for (int64_t u = group0; u < nunits && ok; u += ngroups) {
                int64_t t, uv;
                int ks0, ks1;
                unit_of<SPL>(u, args, nks, t, ks0, ks1, uv);
                int64_t tm64, tc64;
                tile_rc(t, args, tm64, tc64);
                const int tm = (int)tm64;
                const int tn = (int)tc64;
                const int prank = CG == 2 ? (int)crank : 0;        // rank within an MMA pair
                const int a0 = tm * TM * CG + prank * TM;          // this CTA's first A row
                const int b0 = tn * TN * (DT ? 2 : 1) + prank * C::TNB;  // this CTA's first B row
                const bool rev = SERP && args.serp != 0 && ((((u - group0) / ngroups) & 1) != 0);
                const int kbA = ks0 / (KB / KS), kbN = (ks1 + KB / KS - 1) / (KB / KS) - kbA;
                for (int i = 0; i < kbN && ok; ++i, ++itb) {
                    const int kb = rev ? kbA + kbN - 1 - i : kbA + i;
                    const uint32_t bs = itb % NBITS;
                    if (!mbar_wait(&bar->bits_empty[bs], ((itb / NBITS) & 1u) ^ 1u, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    uint8_t *bits = smem + C::SM_BITS + bs * C::BT_BYTES;
                    const int x = (int)(kb * 4);
                    if (ATMA) {
                        mbar_arrive_expect_tx(&bar->bits_full[bs], C::TNB * 32);
                        tma_load_2d(bits + C::BT_B, &tmB, &bar->bits_full[bs], x, b0);
                    } else if (DT) {
                        mbar_arrive_expect_tx(&bar->bits_full[bs], TM * 32 + 2 * C::TNB * 32 + 1024);
                        tma_load_2d(bits + C::BT_A, &tmA, &bar->bits_full[bs], x, a0);
                        tma_load_2d(bits + C::BT_B, &tmB, &bar->bits_full[bs], x, b0);
                        tma_load_2d(bits + C::BT_B1, &tmB, &bar->bits_full[bs], x, b0 + TN);
                        const bool cin = IQP_IN((int64_t)kb * KB + KB - 1, args.mpad, 54);
                        bulk_load(bits + C::BT_CHI, args.chi + (cin ? kb * KB : 0), 512, &bar->bits_full[bs]);
                        bulk_load(bits + C::BT_CLO, args.clo + (cin ? kb * KB : 0), 512, &bar->bits_full[bs]);
                    } else {
                        mbar_arrive_expect_tx(&bar->bits_full[bs], TM * 32 + C::TNB * 32 + 1024);
                        tma_load_2d(bits + C::BT_A, &tmA, &bar->bits_full[bs], x, a0);
                        tma_load_2d(bits + C::BT_B, &tmB, &bar->bits_full[bs], x, b0);
                        // the split of 2 theta is mpad long (bits stages never pass it)
                        const bool cin = IQP_IN((int64_t)kb * KB + KB - 1, args.mpad, 54);
                        bulk_load(bits + C::BT_CHI, args.chi + (cin ? kb * KB : 0), 512, &bar->bits_full[bs]);
                        bulk_load(bits + C::BT_CLO, args.clo + (cin ? kb * KB : 0), 512, &bar->bits_full[bs]);
                    }
                    bmask |= 1u << bs;
                    bpar = (bpar & ~(1u << bs)) | (((itb / NBITS) & 1u) << bs);
                    if (ATMA) {
                        // A_hi / A_lo tiles (W, or a dense operand) of the operand stages of this bits stage.
                        for (int q = 0; q < KB / KS; ++q) {
                            const int ks = kb * (KB / KS) + q;
                            if (ks >= ks1) break;
                            const uint32_t os = ito % NOP;
                            if (!mbar_wait(&bar->op_empty[os], ((ito / NOP) & 1u) ^ 1u, abort_flag, status, lim)) {
                                ok = false;
                                break;
                            }
                            uint8_t *op = smem + C::SM_OP + os * C::OP_BYTES;
                            mbar_arrive_expect_tx(&bar->w_full[os], 2 * TM * KS * 2);
                            tma_load_2d(op + C::OP_A_HI, &tmA, &bar->w_full[os], (int)(ks * KS), a0);
                            tma_load_2d(op + C::OP_A_LO, &tmA2, &bar->w_full[os], (int)(ks * KS), a0);
                            // Warm L2 with the W tiles kWPrefetch stages ahead.
                            if (ks + kWPrefetch < nks) {
                                tma_prefetch_2d(&tmA, (int)((ks + kWPrefetch) * KS), a0);
                                tma_prefetch_2d(&tmA2, (int)((ks + kWPrefetch) * KS), a0);
                            }
                            omask |= 1u << os;
                            opar = (opar & ~(1u << os)) | (((ito / NOP) & 1u) << os);
                            ++ito;
                        }
                    }
                }
            }
            // Drain: every copy this thread issued has landed before exit.
#pragma unroll
            for (int i = 0; i < NBITS; ++i)
                if ((bmask >> i) & 1u) mbar_drain(&bar->bits_full[i], (bpar >> i) & 1u, status, lim);
#pragma unroll
            for (int i = 0; i < NOP; ++i)
                if (ATMA && ((omask >> i) & 1u)) mbar_drain(&bar->w_full[i], (opar >> i) & 1u, status, lim);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0 && leader) {
            uint32_t ito = 0;
            bool ok = true;
            // operand descriptors of stage 0 (K step 0)
            const uint32_t sb = smem_u32(smem + C::SM_OP);
            const uint64_t d_b0 = sdesc_k128(sb + C::OP_B);
            [[maybe_unused]] const uint64_t d_b1 = sdesc_k128(sb + C::OP_B1);
            const uint64_t d_hi0 = sdesc_k128(sb + C::OP_A_HI), d_lo0 = sdesc_k128(sb + C::OP_A_LO);
            for (int64_t u = group0; u < nunits && ok; u += ngroups) {
                int64_t t, uv;
                int ks0, ks1;
                unit_of<SPL>(u, args, nks, t, ks0, ks1, uv);
                int kc = 0;  // stage index within the current accumulation chunk
                for (int ks = ks0; ks < ks1; ++ks, ++ito) {
                    const uint32_t os = ito % NOP;
                    // One-CTA gradient: this thread also waits for the stage's W
                    // tiles (a pair's W halves are vouched for by its producers).
                    const bool got =
                        CG == 2 ? mbar_wait_cluster(&bar->op_full[os], (ito / NOP) & 1u, abort_flag, status, lim)
                                : (mbar_wait(&bar->op_full[os], (ito / NOP) & 1u, abort_flag, status, lim) &&
                                   (!ATMA ||
                                    mbar_wait(&bar->w_full[os], (ito / NOP) & 1u, abort_flag, status, lim)));
                    if (!got) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // first stage of a chunk: overwrite the accumulator
                    const uint32_t acc = kc == 0 ? 0u : 1u;
                    // Descriptors of the stage's first K step (stage os is
                    // os * OP_BYTES / 16 further in the start-address field).
                    const uint64_t so = (uint64_t)(os * (C::OP_BYTES >> 4));
                    // (one function may not mix cta_group::1 and ::2 forms)
                    if constexpr (ATM)
                        umma_stage4_pair_ts(tmem, tmem + kAColBase + os * kAColStage, d_b0 + so, C::IDESC, acc);
                    else if constexpr (DT) {
                        umma_stage4_pair_ss(tmem, d_hi0 + so, d_lo0 + so, d_b0 + so, C::IDESC, acc);
                        umma_stage4_pair_ss(tmem + (uint32_t)TN, d_hi0 + so, d_lo0 + so, d_b1 + so, C::IDESC, acc);
                    } else if constexpr (CG == 2)
                        umma_stage4_pair_ss(tmem, d_hi0 + so, d_lo0 + so, d_b0 + so, C::IDESC, acc);
                    else
                        umma_stage4_ss(tmem, d_hi0 + so, d_lo0 + so, d_b0 + so, C::IDESC, acc);
                    if constexpr (CG == 2) umma_commit_pair(&bar->op_empty[os]);
                    else umma_commit(&bar->op_empty[os]);
                    if (++kc == chunk || ks == ks1 - 1) {
                        if constexpr (CG == 2) umma_commit_pair(&bar->acc_full);
                        else umma_commit(&bar->acc_full);
                        kc = 0;
                    }
                }
            }
            // Drain: all issued MMAs complete before TMEM is freed (and, for a
            // pair, before the peer may leave: the cluster barrier below).
            if constexpr (CG == 2) umma_commit_pair(&bar->drain);
            else umma_commit(&bar->drain);
            mbar_drain(&bar->drain, 0u, status, lim);
        } else if (CG == 2 && lane == 0) {
            // Odd CTA of a pair: forward "my half of stage ks is ready" to the
            // even CTA's stage barrier, one cluster-scope release per stage,
            // so the producer warps themselves only use CTA-scope arrivals.
            const uint32_t op_full_remote = mapa_shared(smem_u32(&bar->op_full[0]), 0u);
            uint32_t ito = 0;
            bool ok = true;
            for (int64_t u = group0; u < nunits && ok; u += ngroups) {
                int64_t t, uv;
                int ks0, ks1;
                unit_of<SPL>(u, args, nks, t, ks0, ks1, uv);
                for (int ks = ks0; ks < ks1; ++ks, ++ito) {
                    const uint32_t os = ito % NOP;
                    if (!mbar_wait(&bar->peer_full[os], (ito / NOP) & 1u, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_remote(op_full_remote + os * 8u);
                }
            }
        }
    } else {
        // ------------------------------------------------ producers + epilogue
        const int gt = threadIdx.x - 64;   // 0 .. NGEN*32-1
        const int quarter = warp & 3;      // TMEM lane quarter this warp may access
        const int group = (warp - 2) >> 2; // accumulator column group of the epilogue
        uint32_t itb = 0, ito = 0, tcount = 0, nacc = 0;
        const int rl = quarter * 32 + lane;  // accumulator row (TMEM lane) of this thread
        // DT: this CTA's running sums (both accumulators) in global memory
        // (the host launches at most kMaxSplitCtas CTAs of this form)
        [[maybe_unused]] float4 *gsum_cta =
            DT && IQP_IN(blockIdx.x, kMaxSplitCtas, 59) ? args.gsum + (int64_t)blockIdx.x * (kDtSumFloats / 4) : nullptr;
        // ATM: this thread's A parity bits of the current bits stage, 16 per
        // operand stage (see expand_a_tmem), packed two stages per word
        uint32_t abits01 = 0, abits23 = 0;
        bool ok = true;
        for (int64_t u = group0; u < nunits && ok; u += ngroups) {
            int ks0, ks1;
            int64_t tm, tc, slot;
            {
                int64_t t;
                unit_of<SPL>(u, args, nks, t, ks0, ks1, slot);
                tile_rc(t, args, tm, tc);
            }
            if (ks0 >= ks1) continue;      // an empty piece of a balanced split: no work
            const uint32_t tix = tcount++;  // units this CTA ran before this one
            const int64_t tn = tc;
            const int64_t arow0 = tm * TM * CG + (CG == 2 ? (int64_t)crank * TM : 0);  // first observable here
            int kc = 0;              // stage index within the current chunk
            int nchunk = 0;          // chunks of this tile already folded into the running sum
            bool fold_due = false;   // a finished chunk must be folded before the next release
            // Stage order: bits stages forwards, or (serpentine rounds) from the
            // last one (c0 operand stages, ks1 - 4 kbTop) down to the first;
            // within a bits stage always q = 0, 1, ...
            const bool rev = SERP && args.serp != 0 && ((((u - group0) / ngroups) & 1) != 0);
            const int kbTop = (ks1 - 1) >> 2;
            const int c0 = ks1 - 4 * kbTop;
            for (int ks = ks0; ks < ks1; ++ks) {
                const int idx = ks - ks0;  // position in the tile's stage sequence
                int q;
                bool qlast;  // the bits stage's last operand stage
                if (!rev) {
                    q = ks & 3;
                    qlast = q == 3 || ks == ks1 - 1;
                } else if (idx < c0) {
                    q = idx;
                    qlast = idx == c0 - 1;
                } else {
                    q = (idx - c0) & 3;
                    qlast = q == 3;
                }
                const uint32_t bs = itb % NBITS;
                if (q == 0 && !wait_warp(&bar->bits_full[bs], (itb / NBITS) & 1u, abort_flag, status, lim)) {
                    ok = false;
                    break;
                }
                const uint8_t *bits = smem + C::SM_BITS + bs * C::BT_BYTES;
                if (ATM && q == 0) {
                    // Row rl's 256 parity bits of this bits stage (8 words);
                    // operand stage j needs bits [64 j + 16 group, +16), in
                    // word 2 j + (group >> 1) at bit 16 (group & 1).
                    const uint4 x0 = *reinterpret_cast<const uint4 *>(bits + C::BT_A + rl * 32);
                    const uint4 x1 = *reinterpret_cast<const uint4 *>(bits + C::BT_A + rl * 32 + 16);
                    const bool odd = (group >> 1) & 1;
                    const uint32_t sh = (uint32_t)(group & 1) * 16u;
                    const uint32_t w0 = odd ? x0.y : x0.x, w1 = odd ? x0.w : x0.z;
                    const uint32_t w2 = odd ? x1.y : x1.x, w3 = odd ? x1.w : x1.z;
                    abits01 = ((w0 >> sh) & 0xFFFFu) | ((w1 >> sh) << 16);
                    abits23 = ((w2 >> sh) & 0xFFFFu) | ((w3 >> sh) << 16);
                }
                const uint32_t os = ito % NOP;
                if (!wait_warp(&bar->op_empty[os], ((ito / NOP) & 1u) ^ 1u, abort_flag, status, lim)) {
                    ok = false;
                    break;
                }
                uint8_t *op = smem + C::SM_OP + os * C::OP_BYTES;
                if (ATM) {
                    // The MMAs that read this stage's A columns have completed
                    // (op_empty); order the TMEM stores after them.
                    tc_fence_after();
                    const uint32_t b16 = ((q < 2 ? abits01 : abits23) >> ((q & 1) * 16)) & 0xFFFFu;
                    const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + kAColBase + os * kAColStage +
                                        (uint32_t)group * 16u;
                    expand_a_tmem(b16, bits + C::BT_CHI, bits + C::BT_CLO, q, group, ta);
                }
                expand_b<C::TNB>(bits + C::BT_B, op + C::OP_B, q, gt);
                if constexpr (DT) expand_b<C::TNB>(bits + C::BT_B1, op + C::OP_B1, q, gt);
                if (!ATMA && !ATM)
                    expand_a(bits + C::BT_A, bits + C::BT_CHI, bits + C::BT_CLO, op + C::OP_A_HI, op + C::OP_A_LO, q,
                             gt);
                if (ATM) {
                    tmem_wait_st();
                    tc_fence_before();
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (ATMA && CG == 2 && !wait_warp(&bar->w_full[os], (ito / NOP) & 1u, abort_flag, status, lim)) {
                    // A pair's W tiles must have landed before the stage is released.
                    ok = false;
                    break;
                }
                if (fold_due) {
                    // This stage opens a new chunk and its first MMA overwrites
                    // the accumulator: fold the finished chunk into the running
                    // sum first, then release the stage (it was produced while
                    // the previous chunk's last MMAs ran).
                    if (!wait_warp(&bar->acc_full, nacc & 1u, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    ++nacc;
                    __syncwarp();
                    tc_fence_after();
                    const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(group * kGroupCols);
#pragma unroll 1
                    for (int c = 0; c < (DT ? 2 : 1) * kGroupLoads; ++c) {
                        uint32_t r[32], acc[32];
                        const int hb = DT && c >= kGroupLoads ? 1 : 0;  // DT: accumulator of the second sample tile
                        const int cc = c - hb * kGroupLoads;
                        tmem_ld32(tb + (uint32_t)(hb * TN + cc * 32), r);
                        if (ATM || DT) {
                            // running sum in shared memory (ATM) or global memory
                            // (DT), this thread's row only
                            float4 *sp = ATM ? sum4 + ((group * kGroupCols + cc * 32) >> 2) * TM + rl
                                             : gsum_cta + ((hb * TN + group * kGroupCols + cc * 32) >> 2) * TM + rl;
#pragma unroll
                            for (int e4 = 0; e4 < 8; ++e4) {
                                float4 v = make_float4(__uint_as_float(r[4 * e4]), __uint_as_float(r[4 * e4 + 1]),
                                                       __uint_as_float(r[4 * e4 + 2]), __uint_as_float(r[4 * e4 + 3]));
                                if (nchunk > 0) {
                                    const float4 o = sp[e4 * TM];
                                    v.x += o.x;
                                    v.y += o.y;
                                    v.z += o.z;
                                    v.w += o.w;
                                }
                                sp[e4 * TM] = v;
                            }
                            continue;
                        }
                        if (nchunk > 0) {
                            tmem_ld32(tb + kSumCol + c * 32, acc);
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                r[e] = __float_as_uint(__uint_as_float(r[e]) + __uint_as_float(acc[e]));
                        }
                        tmem_st32(tb + kSumCol + c * 32, r);
                    }
                    tc_fence_before();
                    ++nchunk;
                    fold_due = false;
                }
                if (lane == 0) {
                    // Even CTA: straight to the stage barrier; odd CTA: to the
                    // local barrier its forwarder watches.
                    if (CG == 2 && !leader) mbar_arrive(&bar->peer_full[os]);
                    else mbar_arrive(&bar->op_full[os]);
                }
                ++ito;
                if (qlast) {
                    if (lane == 0) mbar_arrive(&bar->bits_empty[bs]);
                    ++itb;
                }
                if (++kc == chunk) {
                    kc = 0;
                    fold_due = ks != ks1 - 1;
                }
            }
            if (!ok) break;
            // ------------------------------------------------------ epilogue
            if (!wait_warp(&bar->acc_full, nacc & 1u, abort_flag, status, lim)) {
                ok = false;
                break;
            }
            ++nacc;
            __syncwarp();  // lanes leave the wait loop independently; tcgen05.ld is warp-aligned
            tc_fence_after();
            const int64_t row = arow0 + quarter * 32 + lane;  // observable a
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(group * kGroupCols);
            bool chunked = nchunk > 0;

            if (!GRAD && MODE != 3 && SPL) {
                // A part of a split tile: store this part's accumulator(s);
                // the CTA that finishes the tile's last part sums every
                // part's, in part order, back into TMEM and runs the
                // epilogue. Slot layout: ((slot * CG + CTA) * NH + h) per
                // TM x TN accumulator h (DT: two).
                constexpr int NH = DT ? 2 : 1;
                const int64_t half = CG == 2 ? (int64_t)crank : 0;
                [[maybe_unused]] const int64_t kSkp = args.skcap;  // floats of part scratch
                int64_t tt, np, pbase;  // index among the split tiles, its parts, its first part's slot
                part_info(slot, args, nks, tt, np, pbase);
#pragma unroll 1
                for (int h = 0; h < NH; ++h) {
                    const int64_t so = (((slot * CG + half) * NH + h) * TM + rl) * TN + group * kGroupCols;
                    const float4 *ss0 = ATM  ? sum4 + ((group * kGroupCols) >> 2) * TM + rl
                                        : DT ? gsum_cta + ((h * TN + group * kGroupCols) >> 2) * TM + rl
                                             : nullptr;
                    if (IQP_IN(so + kGroupCols - 1, kSkp, 47))
                        split_store(args.skp + so, tbase + (uint32_t)(h * TN), chunked, ss0);
                }
                __threadfence();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar->part_done);
                const uint32_t nsu = tix;  // split parts this CTA finished before
                if (warp == 2 && lane == 0) {
                    if (mbar_wait(&bar->part_done, nsu & 1u, abort_flag, status, lim)) {
                        int last = 0;
                        if (IQP_IN(tt * CG + half, kMaxSplitCtas, 48)) {
                            int *cnt = args.skc + tt * CG + half;
                            last = atomicAdd(cnt, 1) == np - 1;
                            if (last) {
                                atomicExch(cnt, 0);  // ready for the next launch
                                __threadfence();
                            }
                        }
                        bar->last_flag = last;
                    }
                    mbar_arrive(&bar->part_flag);
                }
                if (!wait_warp(&bar->part_flag, nsu & 1u, abort_flag, status, lim) || *abort_flag) {
                    ok = false;
                    break;
                }
                if (*reinterpret_cast<volatile int *>(&bar->last_flag) == 0) {
                    tc_fence_before();
                    continue;  // another CTA finishes this tile
                }
                __threadfence();
#pragma unroll 1
                for (int h = 0; h < NH; ++h) {
                    const int64_t s0 = (((pbase * CG + half) * NH + h) * TM + rl) * TN + group * kGroupCols;
                    const int64_t pstride = (int64_t)CG * NH * TM * TN;
                    if (IQP_IN(s0 + (np - 1) * pstride + kGroupCols - 1, kSkp, 49))
                        split_sum(args.skp + s0, pstride, (int)np, tbase + (uint32_t)(h * TN));
                }
                chunked = false;  // the sum of the parts is in the accumulator columns
            }
            // Phi (or Q) for 32 columns: last chunk's accumulator + running sum.
            // DT: the two sample tiles' accumulators in turn.
            for (int hb = 0; hb < (DT ? 2 : 1) && ok; ++hb) {
                const int64_t tn_h = DT ? 2 * tn + hb : tn;
                const uint32_t tb_h = tbase + (uint32_t)(hb * TN);
                // where the running sum of this thread's row keeps the group's
                // 32 columns c * 32..: shared memory (ATM), global memory (DT),
                // else TMEM
                auto ssum = [&](int c) -> const float4 * {
                    return ATM  ? sum4 + ((group * kGroupCols + c * 32) >> 2) * TM + rl
                           : DT ? gsum_cta + ((hb * TN + group * kGroupCols + c * 32) >> 2) * TM + rl
                                : nullptr;
                };
                if (!GRAD && MODE == 0) {
                    const int64_t c0 = tn_h * TN + group * kGroupCols;  // first sample of this group
                    int64_t nvalid = args.s - c0;
                    nvalid = nvalid < 0 ? 0 : (nvalid > kGroupCols ? kGroupCols : nvalid);
                    float S = 0.f, M2 = 0.f;
                    uint32_t r[32];
#pragma unroll 1
                    for (int c = 0; c < kGroupLoads; ++c) {
                        load_sum32(tb_h + c * 32, chunked, r, ssum(c));
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (c * 32 + e < nvalid) S += cosf(__uint_as_float(r[e]));
                    }
                    const float mean = nvalid > 0 ? S / (float)nvalid : 0.f;
#pragma unroll 1
                    for (int c = 0; c < kGroupLoads; ++c) {
                        load_sum32(tb_h + c * 32, chunked, r, ssum(c));
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (c * 32 + e < nvalid) {
                                const float d = cosf(__uint_as_float(r[e])) - mean;
                                M2 = fmaf(d, d, M2);
                            }
                    }
                    // Phi itself, when a gradient pass follows (W from it instead
                    // of a second contraction).
                    if (args.out != nullptr) {  // uniform: every lane takes the TMEM loads
#pragma unroll 1
                        for (int c = 0; c * 32 < nvalid; ++c) {
                            load_sum32(tb_h + c * 32, chunked, r, ssum(c));
                            if (row < args.l) store_out32(args, row, c0 + c * 32, r);
                        }
                    }
                    if (row < args.l && nvalid > 0 && IQP_IN(row * args.nparts + c0 / kGroupCols, args.l * args.nparts, 50))
                        args.part[row * args.nparts + (c0 / kGroupCols)] = make_double2((double)S, (double)M2);
                } else if (!GRAD && MODE == 2) {
                    // Both: the statistics of MODE 0 and W of MODE 1 from one
                    // pass over Phi (the loss's alpha, beta known in advance).
                    const int64_t c0 = tn_h * TN + group * kGroupCols;
                    int64_t nvalid = args.s - c0;
                    nvalid = nvalid < 0 ? 0 : (nvalid > kGroupCols ? kGroupCols : nvalid);
                    const bool rv = row < args.l;
                    const float al = rv && IQP_IN(row, args.l, 55) ? (float)args.alpha[row] : 0.f;
                    const float be = (rv && args.beta) ? (float)args.beta[row] : 0.f;
                    float S = 0.f, M2 = 0.f;
                    uint32_t r[32];
#pragma unroll 1
                    for (int c = 0; c < kGroupLoads; ++c) {
                        load_sum32(tb_h + c * 32, chunked, r, ssum(c));
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (c * 32 + e < nvalid) S += cosf(__uint_as_float(r[e]));
                    }
                    const float mean = nvalid > 0 ? S / (float)nvalid : 0.f;
#pragma unroll 1
                    for (int c = 0; c < kGroupLoads; ++c) {
                        load_sum32(tb_h + c * 32, chunked, r, ssum(c));
                        const int64_t i0 = c0 + c * 32;
                        uint32_t ph[16], pl[16];
#pragma unroll
                        for (int e = 0; e < 32; e += 2) {
                            float s0, k0, s1, k1;
                            sincosf(__uint_as_float(r[e]), &s0, &k0);
                            sincosf(__uint_as_float(r[e + 1]), &s1, &k1);
                            const float d0 = k0 - mean, d1 = k1 - mean;
                            if (c * 32 + e < nvalid) M2 = fmaf(d0, d0, M2);
                            if (c * 32 + e + 1 < nvalid) M2 = fmaf(d1, d1, M2);
                            const float w0 = s0 * (al + be * k0), w1 = s1 * (al + be * k1);
                            const float h0 = __bfloat162float(__float2bfloat16_rn(w0));
                            const float h1 = __bfloat162float(__float2bfloat16_rn(w1));
                            ph[e / 2] = pack_bf16x2(h0, h1);
                            pl[e / 2] = pack_bf16x2(w0 - h0, w1 - h1);
                        }
                        if (rv && i0 < args.s) store_w32(args, row, i0, ph, pl);
                    }
                    if (rv && nvalid > 0 && IQP_IN(row * args.nparts + c0 / kGroupCols, args.l * args.nparts, 51))
                        args.part[row * args.nparts + (c0 / kGroupCols)] = make_double2((double)S, (double)M2);
                } else if (!GRAD && MODE == 3) {
                    const int64_t c0 = tn_h * TN + group * kGroupCols;
                    uint32_t r[32];
#pragma unroll 1
                    for (int c = 0; c < kGroupLoads; ++c) {
                        load_sum32(tb_h + c * 32, chunked, r, ssum(c));
                        if (row < args.l && c0 + c * 32 < args.s) store_out32(args, row, c0 + c * 32, r);
                    }
                } else if (!GRAD) {
                    const int64_t c0 = tn_h * TN + group * kGroupCols;
                    const bool rv = row < args.l;
                    const float al = rv && IQP_IN(row, args.l, 55) ? (float)args.alpha[row] : 0.f;
                    const float be = (rv && args.beta) ? (float)args.beta[row] : 0.f;
                    uint32_t r[32];
#pragma unroll 1
                    for (int c = 0; c < kGroupLoads; ++c) {
                        load_sum32(tb_h + c * 32, chunked, r, ssum(c));
                        const int64_t i0 = c0 + c * 32;
                        uint32_t ph[16], pl[16];
#pragma unroll
                        for (int e = 0; e < 32; e += 2) {
                            float s0, k0, s1, k1;
                            sincosf(__uint_as_float(r[e]), &s0, &k0);
                            sincosf(__uint_as_float(r[e + 1]), &s1, &k1);
                            const float w0 = s0 * (al + be * k0), w1 = s1 * (al + be * k1);
                            const float h0 = __bfloat162float(__float2bfloat16_rn(w0));
                            const float h1 = __bfloat162float(__float2bfloat16_rn(w1));
                            ph[e / 2] = pack_bf16x2(h0, h1);
                            pl[e / 2] = pack_bf16x2(w0 - h0, w1 - h1);
                        }
                        if (rv && i0 < args.s) store_w32(args, row, i0, ph, pl);
                    }
                } else {
                    // Gradient epilogue: mask by 2 P_A[a][j], reduce over observables.
                    const bool rv = row < args.l;
                    uint32_t r[32];
#pragma unroll 1
                    for (int c = 0; c < kGroupLoads; ++c) {
                        load_sum32(tb_h + c * 32, chunked, r, ssum(c));
                        const int64_t j0 = tn_h * TN + group * kGroupCols + c * 32;
                        const uint32_t mask = (rv && j0 < args.m &&
                                               IQP_IN(row * args.ldp32 + (j0 >> 5), args.l * args.ldp32, 52))
                                                  ? args.pa32[row * args.ldp32 + (j0 >> 5)]
                                                  : 0u;
                        float v[32];
#pragma unroll
                        for (int e = 0; e < 32; ++e) v[e] = ((mask >> e) & 1u) ? 2.f * __uint_as_float(r[e]) : 0.f;
                        red[quarter * 256 + group * kGroupCols + c * 32 + lane] = reduce_scatter32(v, lane);
                    }
                    // All producer warps' column sums are in `red`; combine the four
                    // lane quarters in fixed order. (The next tile's writes to
                    // `red` follow a full K loop that needs every warp, so a
                    // second barrier is not needed.)
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar->red_full);
                    if (!wait_warp(&bar->red_full, tix & 1u, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    __syncwarp();
                    const int64_t j = tn_h * TN + gt;
                    if (gt < TN && j < args.m && arow0 < args.l) {
                        const double sum = (double)red[gt] + (double)red[256 + gt] + (double)red[512 + gt] +
                                           (double)red[768 + gt];
                        if (IQP_IN((arow0 / TM) * args.m + j, args.tiles_m * args.m, 53))
                            args.gpart[(arow0 / TM) * args.m + j] = sum;
                    }
                }
            }
            if (!ok) break;
            tc_fence_before();
        }
    }

    __syncthreads();
    if (CL == 2) cluster_sync_all();  // no pair MMA still reads the peer's operands
    if (warp == 1) {
        __syncwarp();  // lane 0 ran the MMA loop alone; dealloc is warp-aligned
        tc_fence_after();
        if constexpr (CG == 2) tmem_dealloc_pair(tmem, kTmemCols);
        else tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------------------------ gradient, CTA pairs
// k_grad_pair: the gradient contraction in the transposed orientation,
//   D[j][a] = sum_i S_Z[i][j] W[a][i],   grad partial g_j += sum_a 2 P_A[a][j] D[j][a],
// as CTA pairs (cta_group::2): a tile is 256 gates (M, 128 per CTA) x 256
// observables (N), K = samples in 128-sample operand stages, GNS stages in
// flight.
//  - W (B operand: hi and lo BF16 tiles, 128 observables per CTA, two
//    128-byte K atoms each) arrives by TMA; both CTAs' loads complete on the
//    even CTA's w_full barrier.
//  - S_Z^T (A operand, +-1) is expanded from the transposed sample parities
//    P_Z^T straight into TMEM by eight producer warps (tcgen05.st). The even
//    CTA's producers also wait for the stage's W (w_full, both CTAs' halves)
//    before they arrive, and the odd CTA's readiness is forwarded by one
//    thread, so the MMA thread waits on a single barrier per stage.
//  - The accumulator (256 TMEM columns) is reduced after every accumulation
//    chunk (see below) by eight epilogue warps: mask by 2 P_A[a][j] (bits of
//    P_A^T), sum over the warp's 128 observables in FP32, add into an FP64
//    per-gate partial. Each
//    epilogue warp writes one FP64 partial per (tile, gate): row
//    2 * (observable tile) + (its column half).
// One MMA-issuing thread is the critical path here: its per-stage work is
// one barrier wait and 16 MMAs with precomputed descriptors, and the stage is
// twice as long as the phase kernel's to halve the per-stage overheads.
// Warps: 0 = W loads, 1 = MMA issuer (even CTA) / forwarder (odd CTA),
// 2 = P_Z^T bit loads, 3..10 = producers, 11..18 = epilogue.
// TMEM: accumulator at columns 0..255, A stage os at 256 + 64 os.
constexpr int GN = kGradObs;     // observables per tile (accumulator columns)
constexpr int GNB = GN / 2;      // W rows (observables) per CTA
constexpr int GKS = 128;         // samples per operand stage
constexpr int GNS = 3;           // operand stages in flight
constexpr int GSPB = 256 / GKS;  // operand stages per bits stage
constexpr int GACOLS = GKS / 2;  // TMEM columns per A stage
constexpr int GPROD = 8;         // producer warps
constexpr int GEPI = 8;          // epilogue warps
constexpr int GW0 = 3;           // first producer warp
constexpr int GE0 = GW0 + GPROD; // first epilogue warp
constexpr int kGThreads = (GE0 + GEPI) * 32;
// Accumulation chunks: a tile's K loop is cut into the fewest chunks of at
// most grad_chunk_samples() samples (default 10240), of equal length up to
// one stage. Each chunk boundary stalls the MMAs while the epilogue reads the
// accumulator, so fewer, longer chunks are faster; the chunk bounds the
// error of the tensor core's truncating FP32 accumulation.
constexpr uint32_t kGAcol = GN;      // first A column

struct GCfg {
    static constexpr uint32_t ATOM = GNB * 128;           // one 128-byte K atom of a W tile
    static constexpr uint32_t OP_HI = 0, OP_LO = 2 * ATOM;
    static constexpr uint32_t OP_BYTES = 4 * ATOM;        // W_hi + W_lo, two atoms each
    static constexpr uint32_t SM_BITS = GNS * OP_BYTES;
    static constexpr uint32_t BT_BYTES = TM * 32;         // P_Z^T: 128 gates x 256 samples
    static constexpr uint32_t SM_BAR = SM_BITS + NBITS * BT_BYTES;
    static constexpr uint32_t SM_END = SM_BAR + 256;
    static constexpr uint32_t SMEM = SM_END + 1024;
    static constexpr uint32_t IDESC = idesc_bf16(2 * TM, GN);
    static_assert(OP_BYTES % 1024 == 0 && BT_BYTES % 1024 == 0, "stage alignment");
    static_assert(ATOM == 16384, "umma_stage8_pair_ts_b steps 16384 bytes between K atoms");
    static_assert(kGAcol + GNS * GACOLS <= kTmemCols, "TMEM columns");
    static_assert(SMEM <= 232448, "shared memory");
};

struct GBars {
    uint64_t bits_full[NBITS], bits_empty[NBITS], a_full[GNS], a_peer[GNS], w_full[GNS], empty[GNS], acc_full,
        acc_empty, drain;
    uint32_t tmem_slot;
    int abort_flag;
};

struct GradArgs {
    int64_t l, s, m;
    int64_t nks;                  // operand stages per tile: ceil(s / GKS)
    int64_t chunk;                // operand stages per accumulation chunk
    int64_t tiles_g, tiles_o;     // gate blocks (256), observable blocks (GN)
    int64_t group_o;              // observable blocks per tile group (L2 rasterisation)
    const uint32_t *pat32;        // P_A^T: m rows of ldlt32 32-bit words (bits over observables)
    int64_t ldlt32;
    double *gpart;                // 2 * tiles_o rows of m FP64 partials
    uint32_t *status;
    uint64_t limit_ns;
};

__global__ void __launch_bounds__(kGThreads, 1)
    k_grad_pair(const __grid_constant__ CUtensorMap tmWhi, const __grid_constant__ CUtensorMap tmWlo,
                const __grid_constant__ CUtensorMap tmZt, const GradArgs args) {
    using C = GCfg;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = aligned_smem(smem_raw);
    GBars *bar = reinterpret_cast<GBars *>(smem + C::SM_BAR);
    volatile int *abort_flag = &bar->abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = args.limit_ns;
    uint32_t *status = args.status;
    const uint32_t crank = cluster_ctarank();
    const bool leader = crank == 0;
    const int64_t group0 = blockIdx.x / 2, ngroups = gridDim.x / 2;
    const int64_t ntiles = args.tiles_g * args.tiles_o;
    const int nks = (int)args.nks;
    const int chunk = (int)args.chunk;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NBITS; ++i) {
            mbar_init(&bar->bits_full[i], 1);
            mbar_init(&bar->bits_empty[i], GPROD);
        }
        for (int i = 0; i < GNS; ++i) {
            mbar_init(&bar->a_full[i], GPROD + 1);  // even CTA: its producers + the odd CTA's forwarded arrival
            mbar_init(&bar->a_peer[i], GPROD);     // odd CTA: its producers
            mbar_init(&bar->w_full[i], 1);         // even CTA: its arrive.expect_tx; both CTAs' bytes
            mbar_init(&bar->empty[i], 1);          // the pair commit of the stage's MMAs
        }
        mbar_init(&bar->acc_full, 1);
        mbar_init(&bar->acc_empty, 2 * GEPI);  // even CTA: both CTAs' epilogue warps
        mbar_init(&bar->drain, 1);
        bar->abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async_smem();
    }
    if (warp == 1) {
        tmem_alloc_pair(&bar->tmem_slot, kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = bar->tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ W loads
        if (lane == 0) {
            prefetch_tmap(&tmWhi);
            prefetch_tmap(&tmWlo);
            const uint32_t w_full_leader = mapa_shared(smem_u32(&bar->w_full[0]), 0u);
            uint32_t os = 0, ph = 0, omask = 0, opar = 0;  // stage ring position and its phase parity
            bool ok = true;
            for (int64_t t = group0; t < ntiles && ok; t += ngroups) {
                int64_t to, tg;
                tile_coords(t, args.tiles_o, args.tiles_g, args.group_o, to, tg);
                const int a0 = (int)(to * GN) + (int)crank * GNB;  // this CTA's first W row
                int a0n = -1;                                      // the next tile's (for L2 prefetch)
                if (t + ngroups < ntiles) {
                    int64_t ton, tgn;
                    tile_coords(t + ngroups, args.tiles_o, args.tiles_g, args.group_o, ton, tgn);
                    a0n = (int)(ton * GN) + (int)crank * GNB;
                }
                for (int ks = 0; ks < nks; ++ks) {
                    if (!mbar_wait(&bar->empty[os], ph ^ 1u, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    uint8_t *op = smem + os * C::OP_BYTES;
                    if (leader) mbar_arrive_expect_tx(&bar->w_full[os], 2 * C::OP_BYTES);
#pragma unroll
                    for (int at = 0; at < 2; ++at) {
                        const int x = ks * GKS + at * 64;
                        if (leader) {
                            tma_load_2d(op + C::OP_HI + at * C::ATOM, &tmWhi, &bar->w_full[os], x, a0);
                            tma_load_2d(op + C::OP_LO + at * C::ATOM, &tmWlo, &bar->w_full[os], x, a0);
                        } else {
                            tma_load_2d_pair(op + C::OP_HI + at * C::ATOM, &tmWhi, w_full_leader + os * 8u, x, a0);
                            tma_load_2d_pair(op + C::OP_LO + at * C::ATOM, &tmWlo, w_full_leader + os * 8u, x, a0);
                        }
                    }
                    // warm L2 with the tiles 512 samples beyond this load (the next tile's near the end)
                    int xp = ks * GKS + 512, ap = a0;
                    if (xp >= nks * GKS) {
                        xp -= nks * GKS;
                        ap = a0n;
                    }
                    if (ap >= 0) {
                        tma_prefetch_2d(&tmWhi, xp, ap);
                        tma_prefetch_2d(&tmWhi, xp + 64, ap);
                        tma_prefetch_2d(&tmWlo, xp, ap);
                        tma_prefetch_2d(&tmWlo, xp + 64, ap);
                    }
                    omask |= 1u << os;
                    opar = (opar & ~(1u << os)) | (ph << os);
                    if (++os == GNS) {
                        os = 0;
                        ph ^= 1u;
                    }
                }
            }
            // Drain: every W load has landed before exit (the odd CTA's land on
            // the even CTA's barriers, part of the bytes it expects).
            if (leader) {
#pragma unroll
                for (int i = 0; i < GNS; ++i)
                    if ((omask >> i) & 1u) mbar_drain(&bar->w_full[i], (opar >> i) & 1u, status, lim);
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------------ P_Z^T bit loads
        if (lane == 0) {
            prefetch_tmap(&tmZt);
            uint32_t itb = 0, bmask = 0, bpar = 0;
            bool ok = true;
            for (int64_t t = group0; t < ntiles && ok; t += ngroups) {
                int64_t to, tg;
                tile_coords(t, args.tiles_o, args.tiles_g, args.group_o, to, tg);
                const int j0 = (int)(tg * 2 * TM) + (int)crank * TM;  // this CTA's first gate
                for (int kb = 0; kb < (nks + GSPB - 1) / GSPB; ++kb, ++itb) {
                    const uint32_t bs = itb % NBITS;
                    if (!mbar_wait(&bar->bits_empty[bs], ((itb / NBITS) & 1u) ^ 1u, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    uint8_t *bits = smem + C::SM_BITS + bs * C::BT_BYTES;
                    mbar_arrive_expect_tx(&bar->bits_full[bs], C::BT_BYTES);
                    tma_load_2d(bits, &tmZt, &bar->bits_full[bs], kb * 4, j0);  // 256 samples = 4 words
                    bmask |= 1u << bs;
                    bpar = (bpar & ~(1u << bs)) | (((itb / NBITS) & 1u) << bs);
                }
            }
#pragma unroll
            for (int i = 0; i < NBITS; ++i)
                if ((bmask >> i) & 1u) mbar_drain(&bar->bits_full[i], (bpar >> i) & 1u, status, lim);
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ------------------------------------------------------------ MMA issuer
            uint32_t os = 0, ph = 0, nchk = 0;
            bool ok = true;
            const uint64_t d_w0 = sdesc_k128(smem_u32(smem) + C::OP_HI);  // W_hi of stage 0, K step 0
            for (int64_t t = group0; t < ntiles && ok; t += ngroups) {
                int kc = 0;
                for (int ks = 0; ks < nks; ++ks) {
                    if (kc == 0 &&
                        !mbar_wait_cluster(&bar->acc_empty, (nchk & 1u) ^ 1u, abort_flag, status, lim)) {
                        // the epilogue warps of both CTAs have read the previous chunk
                        ok = false;
                        break;
                    }
                    if (!mbar_wait_cluster(&bar->a_full[os], ph, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t dhi = d_w0 + (uint64_t)(os * (C::OP_BYTES >> 4));
                    umma_stage8_pair_ts_b(tmem, tmem + kGAcol + os * GACOLS, dhi, dhi + (C::OP_LO >> 4), C::IDESC,
                                          kc == 0 ? 0u : 1u);
                    umma_commit_pair(&bar->empty[os]);
                    if (++kc == chunk || ks == nks - 1) {
                        umma_commit_pair(&bar->acc_full);
                        ++nchk;
                        kc = 0;
                    }
                    if (++os == GNS) {
                        os = 0;
                        ph ^= 1u;
                    }
                }
            }
            umma_commit_pair(&bar->drain);
            mbar_drain(&bar->drain, 0u, status, lim);
        } else if (lane == 0) {
            // Odd CTA: forward "my A half of stage os is in TMEM" to the even CTA.
            const uint32_t a_full_remote = mapa_shared(smem_u32(&bar->a_full[0]), 0u);
            uint32_t os = 0, ph = 0;
            bool ok = true;
            for (int64_t t = group0; t < ntiles && ok; t += ngroups) {
                for (int ks = 0; ks < nks; ++ks) {
                    if (!mbar_wait(&bar->a_peer[os], ph, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_remote(a_full_remote + os * 8u);
                    if (++os == GNS) {
                        os = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
    } else if (warp < GE0) {
        // --------------------------------------- producers: S_Z^T (+-1) into TMEM
        const int quarter = warp & 3;        // TMEM lane quarter
        const int h = (warp - GW0) >> 2;     // 64-sample half of each operand stage
        const int rl = quarter * 32 + lane;  // gate row of this CTA
        uint32_t itb = 0, os = 0, ph = 0, zb[4] = {0u, 0u, 0u, 0u};
        bool ok = true;
        for (int64_t t = group0; t < ntiles && ok; t += ngroups) {
            for (int ks = 0; ks < nks; ++ks) {
                const int q = ks % GSPB;
                const uint32_t bs = itb % NBITS;
                if (q == 0) {
                    if (!wait_warp(&bar->bits_full[bs], (itb / NBITS) & 1u, abort_flag, status, lim)) {
                        ok = false;
                        break;
                    }
                    // this row's bits for its halves of the bits stage's two operand stages
                    const uint8_t *bits = smem + C::SM_BITS + bs * C::BT_BYTES;
                    const uint4 x0 = *reinterpret_cast<const uint4 *>(bits + rl * 32);
                    const uint4 x1 = *reinterpret_cast<const uint4 *>(bits + rl * 32 + 16);
                    zb[0] = h ? x0.z : x0.x;  // operand stage 0: words 2 h, 2 h + 1
                    zb[1] = h ? x0.w : x0.y;
                    zb[2] = h ? x1.z : x1.x;  // operand stage 1: words 4 + 2 h, 5 + 2 h
                    zb[3] = h ? x1.w : x1.y;
                }
                if (!wait_warp(&bar->empty[os], ph ^ 1u, abort_flag, status, lim)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + kGAcol + os * GACOLS + (uint32_t)h * 32u;
#pragma unroll
                for (int wd = 0; wd < 2; ++wd) {
                    const uint32_t b = q == 0 ? zb[wd] : zb[2 + wd];
                    uint32_t v[16];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint4 e = expand_pm1((b >> (8 * i)) & 0xFFu);
                        v[4 * i] = e.x;
                        v[4 * i + 1] = e.y;
                        v[4 * i + 2] = e.z;
                        v[4 * i + 3] = e.w;
                    }
                    tmem_st16(ta + (uint32_t)wd * 16u, v);
                }
                tmem_wait_st();
                tc_fence_before();
                // The even CTA's producers vouch for the stage's W as well
                // (both CTAs' halves complete on its w_full).
                if (leader && !wait_warp_cluster(&bar->w_full[os], ph, abort_flag, status, lim)) {
                    ok = false;
                    break;
                }
                __syncwarp();
                if (lane == 0) {
                    if (leader) mbar_arrive(&bar->a_full[os]);
                    else mbar_arrive(&bar->a_peer[os]);
                }
                if (++os == GNS) {
                    os = 0;
                    ph ^= 1u;
                }
                if (q == GSPB - 1 || ks == nks - 1) {
                    if (lane == 0) mbar_arrive(&bar->bits_empty[bs]);
                    ++itb;
                }
            }
        }
    } else {
        // ---------------------------------------------- epilogue: masked reduction
        const int quarter = warp & 3;
        const int e = (warp - GE0) >> 2;  // column half: observables [GNB e, GNB e + GNB) of the tile
        const int rl = quarter * 32 + lane;
        const uint32_t acc_empty_remote = mapa_shared(smem_u32(&bar->acc_empty), 0u);
        constexpr int NW = GNB / 32;
        uint32_t nchk = 0;
        bool ok = true;
        const int nch = (nks + chunk - 1) / chunk;
        for (int64_t t = group0; t < ntiles && ok; t += ngroups) {
            int64_t to, tg;
            tile_coords(t, args.tiles_o, args.tiles_g, args.group_o, to, tg);
            const int64_t j = tg * 2 * TM + (int64_t)crank * TM + rl;  // gate of this thread
            const int64_t a0 = to * GN + (int64_t)e * GNB;             // first observable of this warp
            // 2 P_A[a][j] for the warp's GNB observables: GNB / 32 words of P_A^T
            // row j (a0 is a multiple of 32); bits of observables >= l are dropped.
            uint32_t mk[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) mk[w] = 0u;
            if (j < args.m) {
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int64_t wi = a0 / 32 + w;
                    if (wi < args.ldlt32 && IQP_IN(j * args.ldlt32 + wi, args.m * args.ldlt32, 56))
                        mk[w] = __ldg(args.pat32 + j * args.ldlt32 + wi);
                    const int64_t rem = args.l - (a0 + 32 * w);  // valid observables in this word
                    if (rem < 32) mk[w] &= rem <= 0 ? 0u : ((1u << rem) - 1u);
                }
            }
            double gsum = 0.0;
            for (int c = 0; c < nch; ++c, ++nchk) {
                if (!wait_warp(&bar->acc_full, nchk & 1u, abort_flag, status, lim)) {
                    ok = false;
                    break;
                }
                __syncwarp();
                tc_fence_after();
                float part = 0.f;
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)e * GNB;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    uint32_t r[32];
                    tmem_ld32(tb + w * 32, r);
#pragma unroll
                    for (int x = 0; x < 32; ++x)
                        if ((mk[w] >> x) & 1u) part += __uint_as_float(r[x]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (leader) mbar_arrive(&bar->acc_empty);
                    else mbar_arrive_remote(acc_empty_remote);
                }
                gsum += 2.0 * (double)part;
            }
            if (!ok) break;
            if (j < args.m && IQP_IN((2 * to + e) * args.m + j, 2 * args.tiles_o * args.m, 57))
                args.gpart[(2 * to + e) * args.m + j] = gsum;
        }
    }

    __syncthreads();
    cluster_sync_all();  // no pair MMA or pair-barrier copy still touches the peer
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem, kTmemCols);
    }
}

// Bounded wait on an mbarrier nothing arrives on: exercises the timeout path.
__global__ void k_timeout_selftest(uint32_t *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t b;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&b, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&b, 0u, &abort_flag, status, limit_ns);
    __syncthreads();
}

// ------------------------------------------------------------ tensor maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (fn == nullptr) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Row-major 2D tensor: `cols` elements per row (dim 0), `rows` rows, row
// pitch `pitch_bytes`; box = box_cols x box_rows.
bool make_map(CUtensorMap *map, const void *base, CUtensorMapDataType dt, int64_t cols, int64_t rows,
              int64_t pitch_bytes, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swz) {
    EncodeTiledFn fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(map, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool GRAD, int MODE, int CG, bool AT = GRAD, bool SPL = false, int TA = 0>
cudaError_t launch_k(const CUtensorMap &a, const CUtensorMap &a2, const CUtensorMap &b, const TcArgs &args,
                     cudaStream_t st) {
    using C = Cfg<CG, GRAD || AT, TA == 1 && !GRAD && !AT && CG == 2, TA == 3 && !GRAD && !AT && CG == 2>;
    constexpr int CL = CG;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tc<GRAD, MODE, CG, AT, SPL, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int sms = num_sms();
    if (sms < CL) sms = CL;
    const int64_t groups = args.nunits < sms / CL ? args.nunits : sms / CL;
    LaunchScope ls(GRAD          ? IQP_KERNEL_GRAD_TC
                   : MODE == 1 ? IQP_KERNEL_RECOMPUTE_TC
                   : MODE == 3 ? IQP_KERNEL_LOWORDER_GEMM
                               : IQP_KERNEL_PHASE_TC,
                   st);
    if constexpr (CL == 1) {
        k_tc<GRAD, MODE, 1, AT, SPL, TA><<<(unsigned)groups, kThreads, C::SMEM, st>>>(a, a2, b, args);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(groups * CL), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tc<GRAD, MODE, CG, AT, SPL, TA>, a, a2, b, args);
}

// Tensor-core group size: CTA pairs unless IQP_CTA_PAIRS=0.
// Row blocks per tile group (IQP_TILE_GROUP, 1..64; default 8; 1 = plain
// row-major order).
int64_t tile_group() {
    static int64_t g = -1;
    if (g < 0) {
        const char *e = std::getenv("IQP_TILE_GROUP");
        const long v = e ? std::atol(e) : 8;
        g = (v >= 1 && v <= 64) ? v : 8;
    }
    return g;
}

// Split the last round of phase tiles across idle CTA groups unless
// IQP_SPLIT_TAIL=0.
bool split_tail() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("IQP_SPLIT_TAIL");
        v = (e != nullptr && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Observable blocks per tile group of the pair gradient (IQP_GRAD_GROUP,
// 1..64; default 4). Each block's W panel (256 observables x s samples, hi
// and lo) is read by every gate block of its group; the group's panels must
// stay in L2 while the group sweeps the gate blocks, or W is read from DRAM
// once per round of tiles.
int64_t grad_group() {
    static int64_t g = -1;
    if (g < 0) {
        const char *e = std::getenv("IQP_GRAD_GROUP");
        const long v = e ? std::atol(e) : 4;
        g = (v >= 1 && v <= 64) ? v : 4;
    }
    return g;
}

// Accumulation chunk lengths: gates per chunk of the phase kernels
// (IQP_PHASE_CHUNK, a multiple of 256 from 256 to 65536; default 8192) and
// the longest chunk of the pair gradient in samples (IQP_GRAD_CHUNK, a
// multiple of 128 from 128 to 65536; default 10240). A chunk boundary stalls
// the MMAs while the accumulator is read; a longer chunk lets the tensor
// core's truncating FP32 accumulation drift further. On 10^4 x 10^4 x 10^5
// with theta ~ U(-0.05, 0.05) the gradient's relative error is 1.9e-5 at 4096
// gates, 2.7e-5 at 8192 and 5.3e-5 at 16384; the gradient chunk moves it by
// less than 4e-6 between 2560 and 10240 samples.
int64_t env_multiple(const char *name, int64_t unit, int64_t dflt) {
    const char *e = std::getenv(name);
    const long v = e ? std::atol(e) : dflt;
    return (v >= unit && v <= 65536 && v % unit == 0) ? v : dflt;
}
int64_t phase_chunk_gates() {
    static int64_t g = -1;
    if (g < 0) g = env_multiple("IQP_PHASE_CHUNK", 256, 8192);
    return g;
}
int64_t grad_chunk_samples() {
    static int64_t g = -1;
    if (g < 0) g = env_multiple("IQP_GRAD_CHUNK", 128, 10240);
    return g;
}

// Serpentine gate order for the phase kernels' whole tiles (IQP_PHASE_SERP;
// default 1; 0 = every tile walks the gates forwards).
bool phase_serp() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("IQP_PHASE_SERP");
        v = (e != nullptr && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Phase kernels of CTA pairs: full rounds of tiles of two sample tiles
// (256 observables x 512 samples) against each A stage, the rest as single
// tiles (IQP_PHASE_DT; default 1; 0 = single tiles only).
bool phase_dt() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("IQP_PHASE_DT");
        v = (e != nullptr && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Phase kernels of CTA pairs with the A operand in TMEM (default) or in
// shared memory (IQP_PHASE_TMEM=0).
bool phase_tmem() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("IQP_PHASE_TMEM");
        v = (e != nullptr && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Gradient contraction as CTA pairs in the transposed orientation
// (k_grad_pair, default) or single CTAs (IQP_GRAD_PAIR=0, or IQP_CTA_PAIRS=0).
bool grad_pair() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("IQP_GRAD_PAIR");
        v = (e != nullptr && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

int cta_group() {
    static int cg = -1;
    if (cg < 0) {
        const char *e = std::getenv("IQP_CTA_PAIRS");
        cg = (e != nullptr && e[0] == '0') ? 1 : 2;
    }
    return cg;
}

// Every tile whole (no split parts).
void whole_tiles(TcArgs &a, int64_t ntiles) {
    a.nunits = a.whole = ntiles;
    a.nsplit = 1;
    a.skp = nullptr;
    a.skc = nullptr;
}

template <class T>
T *at(void *ws, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

}  // namespace

namespace {
// Two sample tiles per tile (CTA pairs): whole tiles, or (SPL) the pieces of
// a balanced split of the last round.
template <bool SPL>
cudaError_t launch_phase_dt_k(int mode, const CUtensorMap &ma, const CUtensorMap &mb, const TcArgs &a,
                              cudaStream_t st) {
    if (mode == 0) return launch_k<false, 0, 2, false, SPL, 3>(ma, ma, mb, a, st);
    if (mode == 1) return launch_k<false, 1, 2, false, SPL, 3>(ma, ma, mb, a, st);
    return launch_k<false, 2, 2, false, SPL, 3>(ma, ma, mb, a, st);
}

template <bool SPL>
cudaError_t launch_phase_k(int mode, int cg, const CUtensorMap &ma, const CUtensorMap &mb, const TcArgs &a,
                           cudaStream_t st) {
    if (cg == 2 && phase_tmem()) {
        if (mode == 0) return launch_k<false, 0, 2, false, SPL, 1>(ma, ma, mb, a, st);
        if (mode == 1) return launch_k<false, 1, 2, false, SPL, 1>(ma, ma, mb, a, st);
        return launch_k<false, 2, 2, false, SPL, 1>(ma, ma, mb, a, st);
    }
    if (cg == 2) {
        if (mode == 0) return launch_k<false, 0, 2, false, SPL>(ma, ma, mb, a, st);
        if (mode == 1) return launch_k<false, 1, 2, false, SPL>(ma, ma, mb, a, st);
        return launch_k<false, 2, 2, false, SPL>(ma, ma, mb, a, st);
    }
    if (mode == 0) return launch_k<false, 0, 1, false, SPL>(ma, ma, mb, a, st);
    if (mode == 1) return launch_k<false, 1, 1, false, SPL>(ma, ma, mb, a, st);
    return launch_k<false, 2, 1, false, SPL>(ma, ma, mb, a, st);
}
}  // namespace

cudaError_t launch_phase_tc(int mode, const Plan &p, void *ws, const double *alpha, const double *beta,
                            cudaStream_t st, iqp_status *why) {
    const int cg = cta_group();
    CUtensorMap ma, mb;
    if (!make_map(&ma, at<uint64_t>(ws, p.off_pa), CU_TENSOR_MAP_DATA_TYPE_UINT64, p.ldp, p.l, p.ldp * 8, 4, TM,
                  CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !make_map(&mb, at<uint64_t>(ws, p.off_pz), CU_TENSOR_MAP_DATA_TYPE_UINT64, p.ldp, p.s, p.ldp * 8, 4,
                  (uint32_t)(TN / cg), CU_TENSOR_MAP_SWIZZLE_NONE)) {
        *why = IQP_ERR_UNSUPPORTED;
        return cudaErrorNotSupported;
    }
    TcArgs a{};  // every field zero unless set below
    a.l = p.l;
    a.s = p.s;
    a.m = p.m;
    a.nks = cdiv(p.m, KS);
    a.chunk = phase_chunk_gates() / KS;  // operand stages per accumulation chunk
    a.tiles_m = cdiv(p.l, TM * cg);
    a.tiles_n = cdiv(p.s, TN);
    a.group_m = tile_group();
    a.chi = at<__nv_bfloat16>(ws, p.off_c);
    a.mpad = p.mpad;
    a.clo = a.chi + p.mpad;
    a.part = at<double2>(ws, p.off_part);
    a.nparts = p.nparts;
    a.alpha = alpha;
    a.beta = beta;
    a.whi = at<__nv_bfloat16>(ws, p.off_w);
    a.wlo = a.whi + p.l * p.ldw;
    a.ldw = p.ldw;
    a.pa32 = nullptr;
    a.ldp32 = 2 * p.ldp;
    a.gpart = nullptr;
    // MODE 0 keeps Phi (FP32, l x ldw) when a gradient pass follows.
    a.out = (mode == 0 && p.phi_out) ? static_cast<void *>(p.phi) : nullptr;
    a.ldo = p.ldphi;
    a.out_f64 = 0;
    a.status = at<uint32_t>(ws, p.off_status);
    a.limit_ns = default_spin_limit_ns();
    a.serp = phase_serp() ? 1 : 0;
    // Two sample tiles per tile: the full rounds of double tiles (256 x 512)
    // run in one launch; the double tiles of the last, partial round continue
    // below as single tiles (tile t = half t % 2 of double tile dbase + t / 2).
    int64_t T = a.tiles_m * a.tiles_n;
    {
        int sms = num_sms();
        if (sms > kMaxSplitCtas) sms = kMaxSplitCtas;
        const int64_t P = sms / 2;  // CTA pairs
        const int64_t tiles_n2 = cdiv(p.s, 2 * TN);
        const int64_t T2 = a.tiles_m * tiles_n2;
        if (cg == 2 && phase_dt() && p.off_gsum != 0 && num_sms() <= kMaxSplitCtas && P >= 1 && T2 >= P) {
            const int64_t full = (T2 / P) * P;
            TcArgs d = a;
            d.tiles_n = tiles_n2;
            whole_tiles(d, full);
            d.gsum = at<float4>(ws, p.off_gsum);
            const cudaError_t e = launch_phase_dt_k<false>(mode, ma, mb, d, st);
            if (e != cudaSuccess) return e;
            if (full == T2) return cudaSuccess;
            // The last round, balanced: its double tiles' bits stages, end to
            // end, in P equal ranges, one per CTA pair (pieces of at most two
            // or three tiles each; see unit_of).
            const int64_t left = T2 - full;
            const int64_t nkb = cdiv(a.nks, KB / KS);
            const int64_t W = left * nkb;
            if (split_tail() && p.off_skx != 0 && W >= P && left * 2 <= kMaxSplitCtas) {
                int64_t KP = 1;
                for (int64_t t = 0; t < left; ++t) {
                    const int64_t g0 = ((t * nkb + 1) * P - 1) / W, g1 = ((t + 1) * nkb * P - 1) / W;
                    if (g1 - g0 + 1 > KP) KP = g1 - g0 + 1;
                }
                if (left * KP * 2 * 2 <= kSplitSlots) {
                    TcArgs e2 = d;
                    e2.whole = full;
                    e2.nsplit = 1;
                    e2.nunits = P * (cdiv(W / P + 1, nkb) + 2);
                    e2.sk = 1;
                    e2.skW = W;
                    e2.skP = P;
                    e2.skKP = KP;
                    e2.skp = at<float>(ws, p.off_skx);
                    e2.skc = reinterpret_cast<int *>(e2.skp + (int64_t)kSplitSlots * kSplitSlotFloats);
                    e2.skcap = (int64_t)kSplitSlots * kSplitSlotFloats;
                    const cudaError_t e3 = cudaMemsetAsync(e2.skc, 0, (size_t)(left * 2) * sizeof(int), st);
                    if (e3 != cudaSuccess) return e3;
                    return launch_phase_dt_k<true>(mode, ma, mb, e2, st);
                }
            }
            a.dtmap = 1;
            a.dbase = full;
            a.tiles_n2 = tiles_n2;
            T = 2 * (T2 - full);
        }
    }
    // A last round of tiles that would leave CTA groups idle is split along
    // the gates across them: the whole tiles run first (full rounds), then a
    // second launch runs the remaining tiles' parts, each a range of whole
    // bits stages, and the last part of a tile to finish sums the parts (in
    // part order) and runs the epilogue.
    whole_tiles(a, T);
    int64_t R = 0, ns = 1;
    if (split_tail() && p.off_skp != 0) {
        int sms = num_sms();
        if (sms > kMaxSplitCtas) sms = kMaxSplitCtas;
        const int64_t P = sms / cg;  // CTA groups
        R = T >= P ? T % P : T;
        ns = (P >= 2 && R > 0) ? P / R : 1;
        const int64_t nkb = cdiv(a.nks, KB / KS);
        if (ns > nkb) ns = nkb;
        if (ns < 2) R = 0;
    }
    if (R == 0) return launch_phase_k<false>(mode, cg, ma, mb, a, st);
    if (T - R > 0) {
        TcArgs w = a;
        whole_tiles(w, T - R);
        const cudaError_t e = launch_phase_k<false>(mode, cg, ma, mb, w, st);
        if (e != cudaSuccess) return e;
    }
    a.whole = T - R;
    a.nsplit = (int)ns;
    a.nunits = R * ns;
    a.skp = at<float>(ws, p.off_skp);
    a.skc = reinterpret_cast<int *>(a.skp + (int64_t)kMaxSplitCtas * kSplitSlotFloats);
    a.skcap = (int64_t)kMaxSplitCtas * kSplitSlotFloats;
    const cudaError_t e = cudaMemsetAsync(a.skc, 0, (size_t)(R * cg) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    return launch_phase_k<true>(mode, cg, ma, mb, a, st);
}


namespace {
cudaError_t launch_grad_pair(const Plan &p, void *ws, cudaStream_t st, iqp_status *why) {
    using C = GCfg;
    CUtensorMap mhi, mlo, mz;
    const __nv_bfloat16 *whi = at<__nv_bfloat16>(ws, p.off_w);
    const __nv_bfloat16 *wlo = whi + p.l * p.ldw;
    if (!make_map(&mhi, whi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.s, p.l, p.ldw * 2, KS, GNB,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&mlo, wlo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.s, p.l, p.ldw * 2, KS, GNB,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&mz, at<uint64_t>(ws, p.off_pzt), CU_TENSOR_MAP_DATA_TYPE_UINT64, p.ldzt, p.m, p.ldzt * 8, 4, TM,
                  CU_TENSOR_MAP_SWIZZLE_NONE)) {
        *why = IQP_ERR_UNSUPPORTED;
        return cudaErrorNotSupported;
    }
    GradArgs a;
    a.l = p.l;
    a.s = p.s;
    a.m = p.m;
    a.nks = cdiv(p.s, GKS);
    const int64_t cmax = grad_chunk_samples() / GKS;
    a.chunk = cdiv(a.nks, cdiv(a.nks, cmax));  // fewest chunks, balanced
    a.tiles_g = cdiv(p.m, 2 * TM);
    a.tiles_o = cdiv(p.l, GN);
    a.group_o = grad_group();
    a.pat32 = at<uint32_t>(ws, p.off_pat);
    a.ldlt32 = 2 * p.ldlt;
    a.gpart = at<double>(ws, p.off_gpart);
    a.status = at<uint32_t>(ws, p.off_status);
    a.limit_ns = default_spin_limit_ns();
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_grad_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int sms = num_sms();
    if (sms < 2) sms = 2;
    const int64_t ntiles = a.tiles_g * a.tiles_o;
    const int64_t groups = ntiles < sms / 2 ? ntiles : sms / 2;
    LaunchScope ls(IQP_KERNEL_GRAD_TC, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(groups * 2), 1, 1);
    cfg.blockDim = dim3(kGThreads, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_grad_pair, mhi, mlo, mz, a);
}
}  // namespace

// Rows of FP64 gradient partials the gradient contraction writes: two per
// 256-observable tile for the CTA-pair kernel, one per 128-observable tile
// for the single-CTA kernel (IQP_GRAD_PAIR=0 or IQP_CTA_PAIRS=0).
int64_t grad_tc_rows(const Plan &p) { return cta_group() == 2 && grad_pair() ? 2 * cdiv(p.l, GN) : cdiv(p.l, TM); }

cudaError_t launch_grad_tc(const Plan &p, void *ws, cudaStream_t st, iqp_status *why) {
    if (cta_group() == 2 && grad_pair()) return launch_grad_pair(p, ws, st, why);
    const int cg = 1;
    CUtensorMap mhi, mlo, mb;
    const __nv_bfloat16 *whi = at<__nv_bfloat16>(ws, p.off_w);
    const __nv_bfloat16 *wlo = whi + p.l * p.ldw;
    const uint32_t wrows = TM;
    if (!make_map(&mhi, whi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.s, p.l, p.ldw * 2, KS, wrows,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&mlo, wlo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.s, p.l, p.ldw * 2, KS, wrows,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&mb, at<uint64_t>(ws, p.off_pzt), CU_TENSOR_MAP_DATA_TYPE_UINT64, p.ldzt, p.m, p.ldzt * 8, 4,
                  (uint32_t)(TN / cg), CU_TENSOR_MAP_SWIZZLE_NONE)) {
        *why = IQP_ERR_UNSUPPORTED;
        return cudaErrorNotSupported;
    }
    TcArgs a{};  // every field zero unless set below
    a.l = p.l;
    a.s = p.s;
    a.m = p.m;
    a.nks = cdiv(p.s, KS);
    a.chunk = 32;  // 2048 samples per accumulation chunk
    a.tiles_m = cdiv(p.l, TM * cg);
    a.tiles_n = cdiv(p.m, TN);
    a.group_m = tile_group();
    a.chi = a.clo = nullptr;
    a.mpad = 0;
    a.part = nullptr;
    a.nparts = 0;
    a.alpha = a.beta = nullptr;
    a.whi = a.wlo = nullptr;
    a.ldw = p.ldw;
    a.pa32 = at<uint32_t>(ws, p.off_pa);
    a.ldp32 = 2 * p.ldp;
    a.gpart = at<double>(ws, p.off_gpart);
    a.out = nullptr;
    a.ldo = 0;
    a.out_f64 = 0;
    whole_tiles(a, a.tiles_m * a.tiles_n);
    a.status = at<uint32_t>(ws, p.off_status);
    a.limit_ns = default_spin_limit_ns();
    return launch_k<true, 0, 1>(mhi, mlo, mb, a, st);
}

cudaError_t launch_w_from_phi(const Plan &p, void *ws, const double *alpha, const double *beta, cudaStream_t st) {
    if (p.phi == nullptr || p.ldw % 4 != 0 || p.ldphi % 4 != 0) return cudaErrorInvalidValue;
    __nv_bfloat16 *whi = at<__nv_bfloat16>(ws, p.off_w);
    __nv_bfloat16 *wlo = whi + p.l * p.ldw;
    const int64_t total = p.l * (p.ldw / 4);
    int64_t grid = cdiv(total, 256);
    const int64_t cap = (int64_t)num_sms() * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    LaunchScope ls(IQP_KERNEL_RECOMPUTE_TC, st);
    k_w_from_phi<<<(unsigned)grid, 256, 0, st>>>(p.phi, p.ldphi, p.ldw, p.l, p.s, alpha, beta, whi, wlo);
    return cudaGetLastError();
}

cudaError_t launch_tc_dense(const __nv_bfloat16 *a_hi, const __nv_bfloat16 *a_lo, int64_t rows, int64_t kpad,
                            int64_t k, const uint64_t *b_bits, int64_t nb, int64_t ldb, void *out, int64_t ldo,
                            bool out_f64, uint32_t *status, cudaStream_t st) {
    const int cg = cta_group();
    CUtensorMap mhi, mlo, mb;
    if (kpad % KS != 0 || k > kpad || k > 64 * ldb || ldb % 2 != 0 || ldb < 4 || ldo % 4 != 0 ||
        !make_map(&mhi, a_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, kpad, rows, kpad * 2, KS, TM,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&mlo, a_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, kpad, rows, kpad * 2, KS, TM,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&mb, b_bits, CU_TENSOR_MAP_DATA_TYPE_UINT64, ldb, nb, ldb * 8, 4, (uint32_t)(TN / cg),
                  CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorNotSupported;
    TcArgs a{};  // every field zero unless set below
    a.l = rows;
    a.s = nb;
    a.m = k;
    a.nks = cdiv(k, KS);
    a.chunk = 64;
    a.tiles_m = cdiv(rows, TM * cg);
    a.tiles_n = cdiv(nb, TN);
    a.group_m = tile_group();
    a.chi = a.clo = nullptr;
    a.mpad = 0;
    a.part = nullptr;
    a.nparts = 0;
    a.alpha = a.beta = nullptr;
    a.whi = a.wlo = nullptr;
    a.ldw = 0;
    a.pa32 = nullptr;
    a.ldp32 = 0;
    a.gpart = nullptr;
    a.out = out;
    a.ldo = ldo;
    a.out_f64 = out_f64 ? 1 : 0;
    whole_tiles(a, a.tiles_m * a.tiles_n);
    a.status = status;
    a.limit_ns = default_spin_limit_ns();
    if (cg == 2) return launch_k<false, 3, 2, true>(mhi, mlo, mb, a, st);
    return launch_k<false, 3, 1, true>(mhi, mlo, mb, a, st);
}

cudaError_t launch_timeout_selftest(uint32_t *status, uint64_t limit_ns, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_SELFTEST, st);
    k_timeout_selftest<<<1, 32, 0, st>>>(status, limit_ns);
    return cudaGetLastError();
}

}  // namespace iqp
