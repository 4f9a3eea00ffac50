// GF(2) parity products of Sec. 2.2 (the exponents of B = (-1)^{Z G^T} and
// C = 1 - (-1)^{A G^T}) and the data parity sums of Sec. 3.3.1, on bit-packed
// rows. A lane owns one generator and folds (r AND g) over 32-bit words with
// one LOP3 per word per row into a per-row XOR accumulator; popc(acc) & 1 is
// the parity. Bit-exact.
#include <cstdlib>

#include "common.cuh"
#include "parity.cuh"

namespace iqp {

uint32_t check_word_parity() { return take_check_word(); }

namespace {

constexpr int kRows = 32;    // rows of R per block
constexpr int kGens = 256;   // generators per block (8 warps x 32 lanes)
constexpr int kKW = 32;      // 32-bit words per staged chunk
constexpr int kPad = 36;     // smem row stride in words (16-byte aligned)

// mode 0: P (and optional PT); mode 1: parity sums T.
template <int MODE>
__global__ void __launch_bounds__(256) k_parity(int nw32, const uint32_t *__restrict__ R, int64_t ldr32, int64_t rows,
                                                 const uint32_t *__restrict__ G, int64_t ldg32, int64_t m,
                                                 uint32_t *__restrict__ P, int64_t ldp32, uint32_t *__restrict__ PT,
                                                 int64_t ldpt32, long long *__restrict__ T) {
    __shared__ __align__(16) uint32_t Rs[kRows][kPad];
    __shared__ __align__(16) uint32_t Gs[kGens][kPad];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t g0 = (int64_t)blockIdx.x * kGens;
    const int64_t r0 = (int64_t)blockIdx.y * kRows;
    const int nw4 = (nw32 + 3) & ~3;  // words read per row (padding words are zero)

    uint32_t acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = 0u;

    for (int w0 = 0; w0 < nw4; w0 += kKW) {
        // Stage R chunk: 32 rows x 8 uint4.
        {
            const int row = tid >> 3, q = tid & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (r0 + row < rows && w0 + 4 * q < nw4 && IQP_IN((r0 + row) * ldr32 + w0 + 4 * q + 3, rows * ldr32, 0))
                v = *reinterpret_cast<const uint4 *>(R + (r0 + row) * ldr32 + w0 + 4 * q);
            *reinterpret_cast<uint4 *>(&Rs[row][4 * q]) = v;
        }
        // Stage G chunk: 256 rows x 8 uint4.
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int idx = tid + 256 * k, row = idx >> 3, q = idx & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (g0 + row < m && w0 + 4 * q < nw4 && IQP_IN((g0 + row) * ldg32 + w0 + 4 * q + 3, m * ldg32, 1))
                v = *reinterpret_cast<const uint4 *>(G + (g0 + row) * ldg32 + w0 + 4 * q);
            *reinterpret_cast<uint4 *>(&Gs[row][4 * q]) = v;
        }
        __syncthreads();
        const int kw = min(kKW, nw4 - w0);
        for (int w = 0; w < kw; w += 4) {
            const uint4 g = *reinterpret_cast<const uint4 *>(&Gs[warp * 32 + lane][w]);
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const uint4 rv = *reinterpret_cast<const uint4 *>(&Rs[r][w]);
                acc[r] ^= (rv.x & g.x) ^ (rv.y & g.y) ^ (rv.z & g.z) ^ (rv.w & g.w);
            }
        }
        __syncthreads();
    }

    const int64_t gen = g0 + warp * 32 + lane;
    if (MODE == 0) {
        uint32_t mine = 0u, col = 0u;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const uint32_t bit = __popc(acc[r]) & 1u;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
            if (lane == r) mine = bal;
            col |= bit << r;
        }
        const int64_t row = r0 + lane;
        if (row < rows && (g0 >> 5) + warp < ldp32 && IQP_IN(row * ldp32 + (g0 >> 5) + warp, rows * ldp32, 2))
            P[row * ldp32 + (g0 >> 5) + warp] = mine;
        if (PT != nullptr && gen < m && IQP_IN((r0 >> 5), ldpt32, 3)) PT[gen * ldpt32 + (r0 >> 5)] = col;
    } else {
        // Sum over the valid generators (data rows) of this warp: +1 even, -1 odd.
        int64_t valid = m - (g0 + warp * 32);
        valid = valid < 0 ? 0 : (valid > 32 ? 32 : valid);
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, __popc(acc[r]) & 1u);
            if (lane == r && r0 + r < rows && valid > 0 && IQP_IN(r0 + r, rows, 4)) {
                const long long v = (long long)valid - 2LL * (long long)__popc(bal);
                atomicAdd(reinterpret_cast<unsigned long long *>(T + r0 + r), (unsigned long long)v);
            }
        }
    }
}

// ------------------------------------------------------------------
// Support-gather path. With R^T (n x rows bits) in memory, the parities of
// gate j with 64 consecutive rows are one word:
//   P^T[j][w] = XOR over qubits q in supp(g_j) of R^T[q][w],
// so a generator of weight k costs k coalesced row loads per 64 rows
// (instead of a fold over all n qubits). The row-major P is a bit transpose
// of P^T.

// Bit transpose: out (in_cols x ld_out32*32 bits) = in^T, where in is
// in_rows x in_cols bits with ld_in32 words per row. Output words beyond
// in_rows bits are written as zero; output rows >= in_cols are not written.
// Tile: 512 x 512 bits per block of 512 threads, read and written as
// 64-byte row segments (16-byte accesses where the rows are aligned); each warp transposes 32 x 32 blocks in registers
// (five shuffle stages swapping off-diagonal sub-blocks of 16, 8, 4, 2, 1).
// Batched over blockIdx.y: matrix b starts at in + b in_bs32 / out + b out_bs32.
constexpr int kTT = 512;            // tile edge in bits
constexpr int kTW = kTT / 32;       // 32-bit words per tile row
constexpr int kTPairs = kTW * (kTW + 1) / 2;  // 32 x 32 block pairs (rb <= cb) of a tile

// Block pairs of a tile in the order rb = 0, 1, ..., cb = rb .. kTW - 1.
struct TilePairs {
    uint8_t rb[kTPairs], cb[kTPairs];
};
constexpr TilePairs make_tile_pairs() {
    TilePairs t{};
    int k = 0;
    for (int r = 0; r < kTW; ++r)
        for (int c = r; c < kTW; ++c) {
            t.rb[k] = (uint8_t)r;
            t.cb[k] = (uint8_t)c;
            ++k;
        }
    return t;
}
__constant__ TilePairs kTilePairs = make_tile_pairs();

// Transpose, in place, the 512 x 512-bit tile tin (row r = 16 words, bit b of
// word w = column 32 w + b) as 32 x 32 blocks (row block rb, word column cb):
// each warp takes pairs (rb, cb), (cb, rb) with rb <= cb, transposes both in
// registers and swaps them, so afterwards tin[32 cb + lane][rb] holds row
// 32 cb + lane of the transpose, word rb. A lane stores only to the two words
// it loaded. The 32 x 32 transpose (one row word per lane) takes five
// butterfly rounds j = 16, 8, 4, 2, 1: lane L pairs with lane L ^ j and,
// within every 2j-bit group of its word, keeps its own half (the low half if
// bit j of L is clear: mask m_j; else the high half) and takes the other half
// from the partner's word moved by j bits toward it. The move is a rotation
// by j (lane bit clear: left; set: right), since the bits it wraps around land
// in the half that is kept, so a round is one shuffle, one funnel shift and
// one bitwise select.
__device__ __forceinline__ void transpose_tile_smem(uint32_t (*tin)[kTW + 1], int warp, int lane) {
    uint32_t keep[5], rot[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int j = 16 >> r;
        const uint32_t m = r == 0 ? 0x0000FFFFu : r == 1 ? 0x00FF00FFu : r == 2 ? 0x0F0F0F0Fu
                                                  : r == 3 ? 0x33333333u : 0x55555555u;
        const bool hi = (lane & j) != 0;
        keep[r] = hi ? ~m : m;
        rot[r] = hi ? (uint32_t)(32 - j) : (uint32_t)j;
    }
    for (int item = warp; item < kTPairs; item += kTT / 32) {
        const int rb = kTilePairs.rb[item], cb = kTilePairs.cb[item];
        uint32_t x1 = tin[rb * 32 + lane][cb];
        uint32_t x2 = tin[cb * 32 + lane][rb];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            const int j = 16 >> r;
            const uint32_t y1 = __shfl_xor_sync(0xFFFFFFFFu, x1, j);
            const uint32_t y2 = __shfl_xor_sync(0xFFFFFFFFu, x2, j);
            const uint32_t t1 = __funnelshift_l(y1, y1, rot[r]);
            const uint32_t t2 = __funnelshift_l(y2, y2, rot[r]);
            x1 = (x1 & keep[r]) | (t1 & ~keep[r]);
            x2 = (x2 & keep[r]) | (t2 & ~keep[r]);
        }
        tin[cb * 32 + lane][rb] = x1;
        if (rb != cb) tin[rb * 32 + lane][cb] = x2;
    }
}

// One 512 x 512-bit tile (number bid) of the bit transpose, staged in tin.
__device__ __forceinline__ void bit_transpose_tile(uint32_t (*tin)[kTW + 1], const uint32_t *__restrict__ in,
                                                   int64_t in_rows, int64_t in_cols, int64_t ld_in32,
                                                   uint32_t *__restrict__ out, int64_t ld_out32, int64_t gx,
                                                   int64_t bid) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (bid % gx) * kTT;   // input rows = output bit columns
    const int64_t c0 = (bid / gx) * kTT;   // input bit columns = output rows
    const int64_t w0 = c0 >> 5;
    // Row segments move as 16-byte words (4 threads per 64-byte segment)
    // when the rows are 16-byte aligned, else word by word.
    const bool vin = ((ld_in32 & 3) == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
    {
        uint4 v[kTW / 4];
#pragma unroll
        for (int k = 0; k < kTW / 4; ++k) {
            const int idx = tid + kTT * k, row = idx / 4, q = (idx % 4) * 4;
            const int64_t r = r0 + row;
            if (r < in_rows && !IQP_IN(r * ld_in32 + (w0 + q < ld_in32 ? w0 + q : 0), in_rows * ld_in32, 5)) {
                v[k] = make_uint4(0u, 0u, 0u, 0u);
            } else if (vin && r < in_rows && w0 + q + 3 < ld_in32) {
                v[k] = *reinterpret_cast<const uint4 *>(in + r * ld_in32 + w0 + q);
            } else {
                v[k].x = (r < in_rows && w0 + q < ld_in32) ? in[r * ld_in32 + w0 + q] : 0u;
                v[k].y = (r < in_rows && w0 + q + 1 < ld_in32) ? in[r * ld_in32 + w0 + q + 1] : 0u;
                v[k].z = (r < in_rows && w0 + q + 2 < ld_in32) ? in[r * ld_in32 + w0 + q + 2] : 0u;
                v[k].w = (r < in_rows && w0 + q + 3 < ld_in32) ? in[r * ld_in32 + w0 + q + 3] : 0u;
            }
        }
#pragma unroll
        for (int k = 0; k < kTW / 4; ++k) {
            const int idx = tid + kTT * k, row = idx / 4, q = (idx % 4) * 4;
            tin[row][q] = v[k].x;
            tin[row][q + 1] = v[k].y;
            tin[row][q + 2] = v[k].z;
            tin[row][q + 3] = v[k].w;
        }
    }
    __syncthreads();
    transpose_tile_smem(tin, warp, lane);
    __syncthreads();
    const int64_t ow0 = r0 >> 5;
    const bool vout = ((ld_out32 & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
#pragma unroll
    for (int k = 0; k < kTW / 4; ++k) {
        const int idx = tid + kTT * k, row = idx / 4, q = (idx % 4) * 4;
        const int64_t orow = c0 + row;
        if (orow >= in_cols) continue;
        if (!IQP_IN(orow * ld_out32 + (ow0 + q < ld_out32 ? ow0 + q : 0), in_cols * ld_out32, 6)) continue;
        if (vout && ow0 + q + 3 < ld_out32) {
            *reinterpret_cast<uint4 *>(out + orow * ld_out32 + ow0 + q) =
                make_uint4(tin[row][q], tin[row][q + 1], tin[row][q + 2], tin[row][q + 3]);
        } else {
            for (int e = 0; e < 4; ++e)
                if (ow0 + q + e < ld_out32) out[orow * ld_out32 + ow0 + q + e] = tin[row][q + e];
        }
    }
}

__global__ void __launch_bounds__(kTT) k_bit_transpose(const uint32_t *__restrict__ in, int64_t in_rows,
                                                        int64_t in_cols, int64_t ld_in32,
                                                        uint32_t *__restrict__ out, int64_t ld_out32, int64_t gx,
                                                        int64_t in_bs32, int64_t out_bs32) {
    __shared__ uint32_t tin[kTT][kTW + 1];  // transposed in place
    bit_transpose_tile(tin, in + (int64_t)blockIdx.y * in_bs32, in_rows, in_cols, ld_in32,
                       out + (int64_t)blockIdx.y * out_bs32, ld_out32, gx, blockIdx.x);
}

// Gate j's support entry (q0, q1, q2, |supp g_j|) from its packed row, one thread.
__device__ __forceinline__ int4 support_entry(const uint64_t *__restrict__ row, int64_t n) {
    const int64_t nw = (n + 63) >> 6;
    int cnt = 0, q0 = 0, q1 = 0, q2 = 0;
    for (int64_t w = 0; w < nw; ++w) {
        uint64_t word = row[w];
        if (w == nw - 1 && (n & 63)) word &= (1ull << (n & 63)) - 1ull;  // never a qubit >= n
        while (word) {
            const int q = (int)(64 * w) + __ffsll((long long)word) - 1;
            word &= word - 1ull;
            if (cnt == 0) q0 = q;
            else if (cnt == 1) q1 = q;
            else if (cnt == 2) q2 = q;
            ++cnt;
        }
    }
    return make_int4(q0, q1, q2, cnt);
}

// The parity step's preparation in one launch: two bit transposes of
// different shapes (blocks [0, a.tiles) take the first, the next b.tiles the
// second) and, in the blocks after them, the gates' support list (one gate per
// thread; rows of at most 16 words).
struct BitTransposeJob {
    const uint32_t *in;
    int64_t in_rows, in_cols, ld_in32;
    uint32_t *out;
    int64_t ld_out32, gx, tiles;
};
struct SupportJob {
    const uint64_t *G;
    int64_t m, ldg, n;
    int4 *sup;
};
constexpr int kSlGates = 256;  // gates per support-list block of k_parity_prep
__global__ void __launch_bounds__(kTT) k_parity_prep(BitTransposeJob a, BitTransposeJob b, SupportJob g) {
    __shared__ __align__(16) uint32_t tin[kTT][kTW + 1];  // transposed in place
    const int64_t bid = blockIdx.x;
    if (bid >= a.tiles + b.tiles) {
        // 256 gates: their rows (at most 16 words) staged in tin with coalesced loads, all in flight
        // together (row r at 17 r), then one thread scans each row there
        uint64_t *rows = reinterpret_cast<uint64_t *>(&tin[0][0]);
        static_assert(kSlGates * 17 * 8 <= sizeof(tin), "staged rows");
        const int nw = (int)((g.n + 63) >> 6);
        const int64_t j0 = (bid - a.tiles - b.tiles) * kSlGates;
        uint64_t v[kSlGates * 16 / kTT];
#pragma unroll
        for (int k = 0; k < kSlGates * 16 / kTT; ++k) {
            const int idx = threadIdx.x + kTT * k, r = idx >> 4, w = idx & 15;
            const int64_t j = j0 + r;
            v[k] = (w < nw && j < g.m && IQP_IN(j * g.ldg + w, g.m * g.ldg, 16)) ? g.G[j * g.ldg + w] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < kSlGates * 16 / kTT; ++k) {
            const int idx = threadIdx.x + kTT * k;
            rows[17 * (idx >> 4) + (idx & 15)] = v[k];
        }
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        if (threadIdx.x < kSlGates && j < g.m && IQP_IN(j, g.m, 13))
            g.sup[j] = support_entry(rows + 17 * threadIdx.x, g.n);
        return;
    }
    const bool second = bid >= a.tiles;
    bit_transpose_tile(tin, second ? b.in : a.in, second ? b.in_rows : a.in_rows, second ? b.in_cols : a.in_cols,
                       second ? b.ld_in32 : a.ld_in32, second ? b.out : a.out, second ? b.ld_out32 : a.ld_out32,
                       second ? b.gx : a.gx, bid - (second ? a.tiles : 0));
}

// Support gather and transpose in one pass, one thread per 32 x 32-bit block.
// A CTA of V warps takes 32 V gates x 1024 rows: warp v owns the gates
// g0 + 32 v .. + 31, lane L the row word w = w0 + L (rows 32 w .. 32 w + 31).
// For each of its 32 gates a lane XORs the R^T words at the gate's support
// (the int4 list: first three qubits and the count; a gate with more qubits
// scans its packed row) and stores that P^T word; across the warp these are
// consecutive words of one R^T row and of one P^T row. The lane then
// transposes its 32 words in registers, after which word b holds the 32
// gates' bits of row 32 w + b, one word of P. The words are staged in shared
// memory and the CTA writes P as row segments of V words (the tile's gates),
// so P^T is never read back.
// R^T: n x ldrt32 words (bits over rows, zero past `rows`); P^T: m x ldrt32
// words, all written; P: rows x ldp32 words (bits over gates, zero past m;
// ldp32 a multiple of 4, P 16-byte aligned).
// IT: the index type. int32_t when the host has checked that every element
// index of the launch fits (the common case: fewer instructions per access),
// else int64_t.
constexpr int kGtWords = 32;            // row words per CTA (lanes)
constexpr int kGtRows = 32 * kGtWords;  // 1024 rows per CTA
// Staged P: warp v's 32 lanes x 32 words at gt_region(v) + 33 L + b. The pad
// word per lane puts the 32 lanes of one store (fixed v and b) in 32 distinct
// banks; the offset 32 / (V / 4) per four warps does the same for the loads
// of the output pass, which take four consecutive warps' words of a row.
__host__ __device__ constexpr int gt_region(int V, int v) { return v * 33 * 32 + (32 / (V / 4)) * (v >> 2); }
__host__ __device__ constexpr int gt_staged_words(int V) { return V * 33 * 32 + 32; }
// staged P + support list of a CTA of V warps: 37.9 KB for 8 warps
__host__ __device__ constexpr int gt_smem_bytes(int V) { return gt_staged_words(V) * 4 + 32 * V * 16; }

// Rounds of the in-register 32 x 32 transpose: in every word pair (i, i + J)
// with bit J of i clear, the high J-bit half of each 2J-bit group of x[i]
// trades places with the low half of the same group of x[i + J].
template <int J>
__device__ __forceinline__ void swap_halves(uint32_t (&x)[32], uint32_t lo) {
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if ((i & J) == 0) {
            const uint32_t t = x[i], u = x[i + J];
            // the shifts as multiplies (low and high word), so that they can run beside the selects
            x[i] = (t & lo) | ((u * (1u << J)) & ~lo);
            x[i + J] = (__umulhi(t, 1u << (32 - J)) & lo) | (u & ~lo);
        }
}

// Transpose a 32 x 32-bit block held as 32 words (bit b of x[i] is element
// (i, b)) in place: afterwards bit i of x[b] is the former bit b of x[i].
// In the 16- and 8-bit rounds the halves are whole bytes, and each new word
// is one byte permute of the pair.
__device__ __forceinline__ void transpose32(uint32_t (&x)[32]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t t = x[i], u = x[i + 16];
        x[i] = __byte_perm(t, u, 0x5410);       // low halves of t and u
        x[i + 16] = __byte_perm(t, u, 0x7632);  // high halves
    }
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if ((i & 8) == 0) {
            const uint32_t t = x[i], u = x[i + 8];
            x[i] = __byte_perm(t, u, 0x6240);      // bytes 0 and 2 of t, of u
            x[i + 8] = __byte_perm(t, u, 0x7351);  // bytes 1 and 3
        }
    swap_halves<4>(x, 0x0F0F0F0Fu);
    swap_halves<2>(x, 0x33333333u);
    swap_halves<1>(x, 0x55555555u);
}

// The P^T word of a gate with more than three qubits: the XOR of the R^T
// words (at rtw, pitch ldrt32) of every qubit of its packed row g.
template <typename IT>
__device__ __noinline__ uint32_t gather_wide(const uint64_t *__restrict__ g, IT n, const uint32_t *__restrict__ rtw,
                                             IT ldrt32, int64_t rt_extent) {
    uint32_t v = 0u;
    const IT nw = (n + 63) >> 6;
    for (IT k = 0; k < nw; ++k) {
        uint64_t word = g[k];
        if (k == nw - 1 && (n & 63)) word &= (1ull << (n & 63)) - 1ull;  // never a qubit >= n
        while (word) {
            const IT qb = 64 * k + (IT)__ffsll((long long)word) - 1;
            word &= word - 1ull;
            if (IQP_IN((int64_t)qb * ldrt32, rt_extent, 8)) v ^= rtw[qb * ldrt32];
        }
    }
    return v;
}

// The fast pass over a warp's 32 gates (entries e[0..31]): x[i] = the P^T
// word of gate j0 + i, stored at ptw + i ldrt32 where the lane's word is in
// the row (wok) and, if CHECK, the gate is below jlim = m - j0. It has no
// branch: a gate's three loads are predicated on its weight. The loads of
// gate i + kGtDepth are issued before gate i is combined, so kGtDepth gates'
// loads are in flight behind the latency of the L2.
#ifndef IQP_GT_DEPTH
#define IQP_GT_DEPTH 4  // 2: the same time; 8 (96 registers, half the CTAs per SM): 12% slower
#endif
#ifndef IQP_GT_WARPS_PER_SM
#define IQP_GT_WARPS_PER_SM 32  // the register file's limit at 64 registers per thread
#endif
constexpr int kGtDepth = IQP_GT_DEPTH;
__host__ __device__ constexpr int kGtMinBlocks(int V) { return IQP_GT_WARPS_PER_SM / V; }
template <typename IT, bool CHECK>
__device__ __forceinline__ void gather_fast(uint32_t (&x)[32], const int4 *__restrict__ e,
                                            const uint32_t *__restrict__ rtw, uint32_t *__restrict__ ptw, IT ldrt32,
                                            bool wok, IT jlim, int64_t rt_extent, int64_t pt_at, int64_t pt_extent) {
    constexpr bool kOff = sizeof(IT) == 4;  // entries hold word offsets q ldrt32, else qubits
    uint32_t r0[kGtDepth], r1[kGtDepth], r2[kGtDepth];
    auto issue = [&](int i, int slot) {
        const int4 ei = e[i];  // the same entry for the whole warp
        const IT o0 = kOff ? (IT)ei.x : (IT)ei.x * ldrt32, o1 = kOff ? (IT)ei.y : (IT)ei.y * ldrt32,
                 o2 = kOff ? (IT)ei.z : (IT)ei.z * ldrt32;
        const int c = ei.w & 3;  // the loads past the gate's weight are predicated off: no L1 work
        r0[slot] = c >= 1 && IQP_IN((int64_t)o0, rt_extent, 8) ? rtw[o0] : 0u;
        r1[slot] = c >= 2 && IQP_IN((int64_t)o1, rt_extent, 8) ? rtw[o1] : 0u;
        r2[slot] = c >= 3 && IQP_IN((int64_t)o2, rt_extent, 8) ? rtw[o2] : 0u;
    };
#pragma unroll
    for (int d = 0; d < kGtDepth; ++d) issue(d, d);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int slot = i % kGtDepth;
        const uint32_t v = r0[slot] ^ r1[slot] ^ r2[slot];
        if (i + kGtDepth < 32) issue(i + kGtDepth, slot);
        if (wok && (!CHECK || (IT)i < jlim) && IQP_IN(pt_at + (int64_t)i * ldrt32, pt_extent, 7))
            ptw[(IT)i * ldrt32] = v;
        x[i] = v;
    }
}

// One row matrix of the fused gather: its R^T (n x ldrt32 words), P^T and P,
// and the number of tiles (gx x gy) it takes.
struct GatherSide {
    const uint32_t *RT;
    uint32_t *PT, *P;
    int64_t rows, ldrt32, tiles;
};

// Blocks [0, s0.tiles) take side s0, the rest side s1 (the observables' and
// the samples' parities of one call share the gates and their support list).
template <typename IT, int V>
__global__ void __launch_bounds__(V * 32, kGtMinBlocks(V))
    k_gather_transpose(const int4 *__restrict__ sup, const uint64_t *__restrict__ G, int64_t ldg_, int64_t n_,
                       int64_t m_, GatherSide s0, GatherSide s1, int64_t ldp32_, int64_t gx) {
    const bool second = (int64_t)blockIdx.x >= s0.tiles;
    const uint32_t *__restrict__ RT = second ? s1.RT : s0.RT;
    uint32_t *__restrict__ PT = second ? s1.PT : s0.PT;
    uint32_t *__restrict__ P = second ? s1.P : s0.P;
    const int64_t rows_ = second ? s1.rows : s0.rows, ldrt32_ = second ? s1.ldrt32 : s0.ldrt32;
    static_assert(V == 8 || V == 16, "a CTA row is V words: 2 or 4 16-byte words");
    constexpr int NG = V / 4;  // 16-byte words per staged row
    extern __shared__ __align__(16) uint32_t gt_smem[];
    uint32_t *sP = gt_smem;
    int4 *sS = reinterpret_cast<int4 *>(gt_smem + gt_staged_words(V));  // the tile's support entries
    const IT ldg = (IT)ldg_, n = (IT)n_, m = (IT)m_, rows = (IT)rows_;
    const IT ldrt32 = (IT)ldrt32_, ldp32 = (IT)ldp32_;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t rt_extent = (int64_t)n * ldrt32;
    const int64_t bid = (int64_t)blockIdx.x - (second ? s0.tiles : 0);
    const IT g0 = (IT)((bid % gx) * 32 * V);    // first gate of this tile
    const IT w0 = (IT)((bid / gx) * kGtWords);  // first row word of this tile
    constexpr bool kOff = sizeof(IT) == 4;      // 32-bit word offsets in the entries
    {
        // Each gate's entry for the fast pass: its first three R^T rows and its weight c (1..3); the pass
        // XORs rows 0 .. c - 1. A gate with no qubit or more than three is marked by 4 and redone from its
        // packed row after the fast pass; gates past m get zero words (weight 0). Rows are given as word
        // offsets (q ldrt32) where those fit in 32 bits, else as qubits.
        const IT j = g0 + tid;
        const IT pitch = kOff ? ldrt32 : (IT)1;
        int4 e = make_int4(0, 0, 0, 0);
        if (j < m && IQP_IN(j, m, 14)) {
            const int4 sp = sup[j];
            const int o0 = (int)((IT)sp.x * pitch), o1 = (int)((IT)sp.y * pitch), o2 = (int)((IT)sp.z * pitch);
            e = sp.w >= 1 && sp.w <= 3 ? make_int4(o0, o1, o2, sp.w) : make_int4(0, 0, 0, 4);
        }
        sS[tid] = e;
    }
    __syncthreads();
    // Lanes past the row read in bounds; their words are never stored: the P rows they would form lie past
    // `rows` (32 ldrt32 >= rows).
    const IT w = w0 + lane;
    const bool wok = w < ldrt32;
    const uint32_t *rtw = RT + (wok ? w : 0);
    uint32_t x[32];
    {
        const IT j0 = g0 + 32 * warp;
        uint32_t *ptw = PT + (wok && j0 < m ? j0 * ldrt32 + w : 0);  // dereferenced only for gates below m
        const int64_t pt_at = (int64_t)j0 * ldrt32 + w, pt_extent = (int64_t)m * ldrt32;
        if (j0 + 32 <= m)  // every gate of the warp is below m
            gather_fast<IT, false>(x, sS + 32 * warp, rtw, ptw, ldrt32, wok, m - j0, rt_extent, pt_at, pt_extent);
        else
            gather_fast<IT, true>(x, sS + 32 * warp, rtw, ptw, ldrt32, wok, m - j0, rt_extent, pt_at, pt_extent);
    }
    const uint32_t wide = __ballot_sync(0xFFFFFFFFu, sS[32 * warp + lane].w == 4);
    if (wide != 0u) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if ((wide >> i) & 1u) {
                const IT j = g0 + 32 * warp + i;  // < m: entries past m are never marked
                const uint32_t v = IQP_IN((int64_t)j * ldg, (int64_t)m * ldg, 15)
                                       ? gather_wide<IT>(G + j * ldg, n, rtw, ldrt32, rt_extent)
                                       : 0u;
                if (wok && IQP_IN((int64_t)j * ldrt32 + w, (int64_t)m * ldrt32, 7)) PT[j * ldrt32 + w] = v;
                x[i] = v;
            }
    }
    transpose32(x);
    {
        uint32_t *col = sP + gt_region(V, warp) + 33 * lane;
#pragma unroll
        for (int b = 0; b < 32; ++b) col[b] = x[b];
    }
    __syncthreads();
    // Thread t writes 16-byte word t % NG of the tile's row t / NG + 128 k.
    const int grp = tid % NG;
    const IT c = (g0 >> 5) + 4 * grp;
    if (c >= ldp32) return;  // ldp32 and c are multiples of 4: whole 16-byte words
    const uint32_t *src = sP + gt_region(V, 4 * grp);  // warps 4 grp .. + 3 share the offset of gt_region
#pragma unroll
    for (int k = 0; k < kGtRows / 128; ++k) {
        const int r = tid / NG + 128 * k;  // row of the tile: lane r / 32, word r % 32
        const IT row = 32 * w0 + r;
        if (row >= rows) break;
        const int pos = r + (r >> 5);
        const uint4 o = make_uint4(src[pos], src[33 * 32 + pos], src[2 * 33 * 32 + pos], src[3 * 33 * 32 + pos]);
        if (IQP_IN((int64_t)row * ldp32 + c + 3, (int64_t)rows * ldp32, 9))
            *reinterpret_cast<uint4 *>(P + row * ldp32 + c) = o;
    }
}

// P^T[j][w] = XOR_{q in supp(g_j)} RT[q][w] for w < ldpt. One warp per
// (gate, 256-word tile); the gate's support is scanned from its packed row.
__global__ void __launch_bounds__(256) k_support_gather(const uint64_t *__restrict__ G, int64_t m, int64_t ldg,
                                                         int64_t n, const uint64_t *__restrict__ RT, int64_t ldrt,
                                                         uint64_t *__restrict__ PT, int64_t ldpt) {
    const int nw = (int)((n + 63) >> 6);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 8 + warp;
    if (j >= m) return;
    const int64_t wt = (int64_t)blockIdx.y * 256;
    uint64_t acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0ull;
    for (int wb = 0; wb < nw; wb += 32) {
        const uint64_t word = (wb + lane < nw) ? G[j * ldg + wb + lane] : 0ull;
        uint32_t nz = __ballot_sync(0xFFFFFFFFu, word != 0ull);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1u;
            uint64_t wv = __shfl_sync(0xFFFFFFFFu, word, src);
            while (wv) {
                const int b = __ffsll((long long)wv) - 1;
                wv &= wv - 1ull;
                const int64_t q = (int64_t)64 * (wb + src) + b;
                if (q >= n) break;  // padding bits must be zero; never read past R^T
                if (!IQP_IN(q * ldrt + wt, n * ldrt, 10)) continue;
                const uint64_t *rt = RT + q * ldrt + wt;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int64_t w = lane + 32 * k;
                    if (wt + w < ldpt) acc[k] ^= rt[w];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int64_t w = wt + lane + 32 * k;
        if (w < ldpt && IQP_IN(j * ldpt + w, m * ldpt, 11)) PT[j * ldpt + w] = acc[k];
    }
}

cudaError_t bit_transpose(const uint64_t *in, int64_t in_rows, int64_t in_cols, int64_t ld_in, uint64_t *out,
                          int64_t ld_out, cudaStream_t st) {
    const int64_t gx = cdiv(ld_out * 64, kTT);
    const int64_t gy = cdiv(in_cols, kTT);
    if (gx * gy > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    LaunchScope ls(IQP_KERNEL_PARITY, st);
    k_bit_transpose<<<(unsigned)(gx * gy), kTT, 0, st>>>(reinterpret_cast<const uint32_t *>(in), in_rows, in_cols,
                                                          2 * ld_in, reinterpret_cast<uint32_t *>(out), 2 * ld_out, gx,
                                                          0, 0);
    return cudaGetLastError();
}

// Support list of every generator: (q0, q1, q2, |supp g_j|), the first three
// qubits of its support in increasing order. One warp per generator.
__global__ void __launch_bounds__(256) k_support_list(const uint64_t *__restrict__ G, int64_t m, int64_t ldg,
                                                       int64_t n, int4 *__restrict__ sup) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= m) return;
    const int64_t nw = (n + 63) >> 6;
    int cnt = 0, q0 = 0, q1 = 0, q2 = 0;
    for (int64_t wb = 0; wb < nw; wb += 32) {
        const uint64_t word = (wb + lane < nw) ? G[j * ldg + wb + lane] : 0ull;
        uint32_t nz = __ballot_sync(0xFFFFFFFFu, word != 0ull);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1u;
            uint64_t wv = __shfl_sync(0xFFFFFFFFu, word, src);
            while (wv) {
                const int b = __ffsll((long long)wv) - 1;
                wv &= wv - 1ull;
                const int64_t q = 64 * (wb + src) + b;
                if (q >= n) break;
                if (cnt == 0) q0 = (int)q;
                else if (cnt == 1) q1 = (int)q;
                else if (cnt == 2) q2 = (int)q;
                ++cnt;
            }
        }
    }
    if (lane == 0 && IQP_IN(j, m, 12)) sup[j] = make_int4(q0, q1, q2, cnt);
}

// The same list with one thread per generator, for rows of at most 16 words
// (n <= 1024): a warp per generator would leave most lanes idle there.
__global__ void __launch_bounds__(256) k_support_list_short(const uint64_t *__restrict__ G, int64_t m, int64_t ldg,
                                                             int64_t n, int4 *__restrict__ sup) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        if (IQP_IN(j, m, 13)) sup[j] = support_entry(G + j * ldg, n);
}

}  // namespace

// Transposes `batch` bit matrices of in_rows x in_cols bits (ld_in words per
// row, consecutive in memory) into in_cols x (64 ld_out) bits each, also
// consecutive: matrix b of the output starts at out + b in_cols ld_out.
cudaError_t launch_bit_transpose_batched(const uint64_t *in, int64_t batch, int64_t in_rows, int64_t in_cols,
                                         int64_t ld_in, uint64_t *out, int64_t ld_out, cudaStream_t st) {
    const int64_t gx = cdiv(ld_out * 64, kTT);
    const int64_t gy = cdiv(in_cols, kTT);
    if (gx * gy > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
        const int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
        LaunchScope ls(IQP_KERNEL_PARITY, st);
        k_bit_transpose<<<dim3((unsigned)(gx * gy), (unsigned)nb), kTT, 0, st>>>(
            reinterpret_cast<const uint32_t *>(in + b0 * in_rows * ld_in), in_rows, in_cols, 2 * ld_in,
            reinterpret_cast<uint32_t *>(out + b0 * in_cols * ld_out), 2 * ld_out, gx, 2 * in_rows * ld_in,
            2 * in_cols * ld_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_support_list(const uint64_t *G, int64_t m, int64_t ldg, int64_t n, int4 *sup, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_PARITY, st);
    if (cdiv(n, 64) <= 16) {
        int64_t blocks = cdiv(m, 256);
        if (blocks > 16384) blocks = 16384;
        k_support_list_short<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(G, m, ldg, n, sup);
    } else {
        k_support_list<<<(unsigned)cdiv(m, 8), 256, 0, st>>>(G, m, ldg, n, sup);
    }
    return cudaGetLastError();
}

// Warps per CTA of the fused gather (IQP_GATHER_WARPS, 8 or 16; default 8:
// four CTAs per SM, whose phases interleave better than two CTAs of 16).
int gather_warps() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("IQP_GATHER_WARPS");
        v = (e != nullptr && std::atoi(e) == 16) ? 16 : 8;
    }
    return v;
}

template <int V>
cudaError_t launch_gather_transpose(bool i32, int64_t gx, const int4 *sup, const uint64_t *G, int64_t ldg, int64_t n,
                                    int64_t m, const GatherSide &s0, const GatherSide &s1, int64_t ldp32,
                                    cudaStream_t st) {
    constexpr int smem = gt_smem_bytes(V);
    static bool attr_set[2] = {false, false};
    if (!attr_set[i32]) {
        const cudaError_t e =
            i32 ? cudaFuncSetAttribute(k_gather_transpose<int32_t, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem)
                : cudaFuncSetAttribute(k_gather_transpose<int64_t, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
        if (e != cudaSuccess) return e;
        attr_set[i32] = true;
    }
    const int64_t blocks = s0.tiles + s1.tiles;
    if (blocks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    LaunchScope ls(IQP_KERNEL_PARITY, st);
    if (i32)
        k_gather_transpose<int32_t, V><<<(unsigned)blocks, V * 32, smem, st>>>(sup, G, ldg, n, m, s0, s1, ldp32, gx);
    else
        k_gather_transpose<int64_t, V><<<(unsigned)blocks, V * 32, smem, st>>>(sup, G, ldg, n, m, s0, s1, ldp32, gx);
    return cudaGetLastError();
}

cudaError_t launch_parity_gather_fused(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, int4 *sup,
                                       bool form_sup, int64_t ldp, const ParitySide *side, int nside,
                                       cudaStream_t st) {
    if (nside < 1 || nside > 2 || ldp % 2 != 0) return cudaErrorInvalidValue;
    // the support list in the preparation launch where its rows are short, else on its own first
    const bool sup_in_prep = form_sup && cdiv(n, 64) <= 16;
    if (form_sup && !sup_in_prep) {
        const cudaError_t e = launch_support_list(G, m, ldg, n, sup, st);
        if (e != cudaSuccess) return e;
    }
    BitTransposeJob bt[2] = {};
    for (int k = 0; k < nside; ++k) {
        const ParitySide &d = side[k];
        bt[k] = BitTransposeJob{reinterpret_cast<const uint32_t *>(d.R), d.rows, n, 2 * d.ldr,
                                reinterpret_cast<uint32_t *>(d.RT), 2 * d.ldpt, cdiv(d.ldpt * 64, kTT), 0};
        bt[k].tiles = bt[k].gx * cdiv(n, kTT);
    }
    const int64_t sl_blocks = sup_in_prep ? cdiv(m, kSlGates) : 0;
    if (bt[0].tiles + bt[1].tiles + sl_blocks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    {
        LaunchScope ls(IQP_KERNEL_PARITY, st);
        k_parity_prep<<<(unsigned)(bt[0].tiles + bt[1].tiles + sl_blocks), kTT, 0, st>>>(
            bt[0], bt[1], SupportJob{G, m, ldg, n, sup});
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // The tiles cover every word of P (gates past m give zero words) and of P^T.
    const int V = gather_warps(), tg = 32 * V;  // gates per tile
    int64_t gx = cdiv(m, tg);
    if (gx < cdiv(2 * ldp, tg / 32)) gx = cdiv(2 * ldp, tg / 32);
    GatherSide gs[2] = {};
    const int64_t lim = (int64_t)1 << 31;
    bool i32 = m * ldg < lim && gx * tg < lim;  // 32-bit element indices where every one of the launch fits
    for (int k = 0; k < nside; ++k) {
        const ParitySide &d = side[k];
        const int64_t gy = cdiv(2 * d.ldpt, kGtWords);
        gs[k] = GatherSide{reinterpret_cast<const uint32_t *>(d.RT), reinterpret_cast<uint32_t *>(d.PT),
                           reinterpret_cast<uint32_t *>(d.P), d.rows, 2 * d.ldpt, gx * gy};
        i32 = i32 && m * 2 * d.ldpt < lim && d.rows * 2 * ldp < lim && n * 2 * d.ldpt < lim && gy * kGtRows < lim;
    }
    if (V == 16) return launch_gather_transpose<16>(i32, gx, sup, G, ldg, n, m, gs[0], gs[1], 2 * ldp, st);
    return launch_gather_transpose<8>(i32, gx, sup, G, ldg, n, m, gs[0], gs[1], 2 * ldp, st);
}

// Support-gather parities: RT (n x ldpt words) is scratch; writes PT
// (m x ldpt words: bits over rows, zero beyond `rows`) and, if P != nullptr,
// P (rows x ldp words: bits over gates, zero beyond m). With the gates'
// support list `sup` (and ldp even) P^T and P come from one fused pass;
// without it P^T is gathered, then transposed into P.
cudaError_t launch_parity_gather(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr, const uint64_t *G,
                                 int64_t m, int64_t ldg, uint64_t *P, int64_t ldp, uint64_t *PT, int64_t ldpt,
                                 uint64_t *RT, cudaStream_t st, const int4 *sup) {
    if (sup != nullptr && P != nullptr && ldp % 2 == 0) {
        // with the gates' support list (launch_support_list): P^T and P from one pass
        const ParitySide side{R, rows, ldr, P, PT, ldpt, RT};
        return launch_parity_gather_fused(n, G, m, ldg, const_cast<int4 *>(sup), false, ldp, &side, 1, st);
    }
    cudaError_t e = bit_transpose(R, rows, n, ldr, RT, ldpt, st);
    if (e != cudaSuccess) return e;
    {
        dim3 grid((unsigned)cdiv(m, 8), (unsigned)cdiv(ldpt, 256));
        LaunchScope ls(IQP_KERNEL_PARITY, st);
        k_support_gather<<<grid, 256, 0, st>>>(G, m, ldg, n, RT, ldpt, PT, ldpt);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (P != nullptr) return bit_transpose(PT, m, rows, ldpt, P, ldp, st);
    return cudaSuccess;
}

// P (rows x ldp words) and, if PT != nullptr, P^T (m x ldpt words). Every
// word of every P row is written (bits >= m are zero); PT rows get the bits
// of rows [0, row_words*64) where row_words = ldpt if PT else ceil(rows/64).
cudaError_t launch_parity(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr, const uint64_t *G, int64_t m,
                          int64_t ldg, uint64_t *P, int64_t ldp, uint64_t *PT, int64_t ldpt, cudaStream_t st) {
    const int nw32 = (int)(2 * cdiv(n, 64));
    const int64_t gx = cdiv(ldp * 64, kGens);
    const int64_t ry = PT ? ldpt * 2 : cdiv(rows, kRows);
    for (int64_t y0 = 0; y0 < ry; y0 += 65535) {
        const int64_t ny = ry - y0 < 65535 ? ry - y0 : 65535;
        dim3 grid((unsigned)gx, (unsigned)ny);
        const int64_t roff = y0 * kRows;
        const int64_t rrows = rows - roff;
        LaunchScope ls(IQP_KERNEL_PARITY, st);
        k_parity<0><<<grid, 256, 0, st>>>(nw32, reinterpret_cast<const uint32_t *>(R + roff * ldr), 2 * ldr,
                                          rrows, reinterpret_cast<const uint32_t *>(G), 2 * ldg, m,
                                          reinterpret_cast<uint32_t *>(P + roff * ldp), 2 * ldp,
                                          PT ? reinterpret_cast<uint32_t *>(PT) + (roff >> 5) : nullptr, 2 * ldpt,
                                          nullptr);
    }
    return cudaGetLastError();
}

// T[a] = sum_x (-1)^{a.x}; T is zeroed here.
cudaError_t launch_parity_sum(int64_t n, const uint64_t *A, int64_t l, int64_t lda, const uint64_t *X, int64_t N,
                              int64_t ldx, int64_t *T, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(T, 0, sizeof(int64_t) * (size_t)l, st);
    if (e != cudaSuccess) return e;
    const int nw32 = (int)(2 * cdiv(n, 64));
    const int64_t gx = cdiv(N, kGens);
    const int64_t ry = cdiv(l, kRows);
    for (int64_t y0 = 0; y0 < ry; y0 += 65535) {
        const int64_t ny = ry - y0 < 65535 ? ry - y0 : 65535;
        const int64_t roff = y0 * kRows;
        dim3 grid((unsigned)gx, (unsigned)ny);
        LaunchScope ls(IQP_KERNEL_PARITY_SUM, st);
        k_parity<1><<<grid, 256, 0, st>>>(nw32, reinterpret_cast<const uint32_t *>(A + roff * lda), 2 * lda,
                                          l - roff, reinterpret_cast<const uint32_t *>(X), 2 * ldx, N, nullptr, 0,
                                          nullptr, 0, reinterpret_cast<long long *>(T + roff));
    }
    return cudaGetLastError();
}

}  // namespace iqp
