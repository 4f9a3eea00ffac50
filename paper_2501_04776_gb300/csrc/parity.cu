// GF(2) parity products of Sec. 2.2 (the exponents of B = (-1)^{Z G^T} and
// C = 1 - (-1)^{A G^T}) and the data parity sums of Sec. 3.3.1, on bit-packed
// rows. A lane owns one generator and folds (r AND g) over 32-bit words with
// one LOP3 per word per row into a per-row XOR accumulator; popc(acc) & 1 is
// the parity. Bit-exact.
#include "common.cuh"

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

__global__ void __launch_bounds__(kTT) k_bit_transpose(const uint32_t *__restrict__ in, int64_t in_rows,
                                                        int64_t in_cols, int64_t ld_in32,
                                                        uint32_t *__restrict__ out, int64_t ld_out32, int64_t gx,
                                                        int64_t in_bs32, int64_t out_bs32) {
    in += (int64_t)blockIdx.y * in_bs32;
    out += (int64_t)blockIdx.y * out_bs32;
    __shared__ uint32_t tin[kTT][kTW + 1];  // transposed in place
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t bid = blockIdx.x;
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

// Support gather and transpose in one pass: for a tile of 512 gates x 512
// rows, each P^T word is formed from the gates' supports (int4 list: first
// three qubits and the count; gates with more than three qubits scan their
// packed row) as the XOR of R^T rows, written to P^T, and the tile is
// transposed in shared memory (as in k_bit_transpose) and written to P, so
// P^T is never read back. R^T: n x ldrt32 words (bits over rows, zero past
// `rows`); P^T: m x ldpt32 words; P: rows x ldp32 words (bits over gates,
// zero past m).
// IT: the index type. int32_t when the host has checked that every element
// index of the launch fits (the common case: fewer instructions per access),
// else int64_t.
template <typename IT>
__global__ void __launch_bounds__(kTT) k_gather_transpose(const int4 *__restrict__ sup, const uint64_t *__restrict__ G,
                                                           int64_t ldg_, int64_t n_, int64_t m_, int64_t rows_,
                                                           const uint32_t *__restrict__ RT, int64_t ldrt32_,
                                                           uint32_t *__restrict__ PT, int64_t ldpt32_,
                                                           uint32_t *__restrict__ P, int64_t ldp32_, int64_t gx) {
    __shared__ uint32_t tin[kTT][kTW + 1];
    const IT ldg = (IT)ldg_, n = (IT)n_, m = (IT)m_, rows = (IT)rows_;
    const IT ldrt32 = (IT)ldrt32_, ldpt32 = (IT)ldpt32_, ldp32 = (IT)ldp32_;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t bid = blockIdx.x;
    const IT r0 = (IT)((bid % gx) * kTT);  // gates (P^T rows) of this tile
    const IT c0 = (IT)((bid / gx) * kTT);  // rows (P^T bit columns) of this tile
    const IT w0 = c0 >> 5;
    // this thread's rows of the tile are row0 + kTT / 4 * k, its words q .. q + 3
    const int row0 = tid / 4, q = (tid % 4) * 4;
    const bool colok = w0 + q < ldrt32;
    const uint32_t *rtq = RT + w0 + q;  // + qubit * ldrt32
#pragma unroll
    for (int k = 0; k < kTW / 4; ++k) {
        const int row = row0 + (kTT / 4) * k;
        const IT j = r0 + row;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (j < m && colok && IQP_IN((int64_t)j * ldpt32 + w0 + q + 3, (int64_t)m * ldpt32, 7)) {
            const int4 sp = sup[j];
            if (sp.w <= 3 && IQP_IN(sp.w > 0 ? sp.x : 0, n, 8) && IQP_IN(sp.w > 1 ? sp.y : 0, n, 8) &&
                IQP_IN(sp.w > 2 ? sp.z : 0, n, 8)) {
                // ldrt32 is a multiple of 8 and w0 + q of 4: the 16-byte word is inside the row
                if (sp.w > 0) {
                    const uint4 a = *reinterpret_cast<const uint4 *>(rtq + (IT)sp.x * ldrt32);
                    v.x ^= a.x; v.y ^= a.y; v.z ^= a.z; v.w ^= a.w;
                }
                if (sp.w > 1) {
                    const uint4 a = *reinterpret_cast<const uint4 *>(rtq + (IT)sp.y * ldrt32);
                    v.x ^= a.x; v.y ^= a.y; v.z ^= a.z; v.w ^= a.w;
                }
                if (sp.w > 2) {
                    const uint4 a = *reinterpret_cast<const uint4 *>(rtq + (IT)sp.z * ldrt32);
                    v.x ^= a.x; v.y ^= a.y; v.z ^= a.z; v.w ^= a.w;
                }
            } else if (sp.w > 3) {
                // every qubit of the support, from the packed row
                const IT nw = (n + 63) >> 6;
                for (IT w = 0; w < nw; ++w) {
                    uint64_t word = G[j * ldg + w];
                    if (w == nw - 1 && (n & 63)) word &= (1ull << (n & 63)) - 1ull;
                    while (word) {
                        const IT qb = 64 * w + (IT)__ffsll((long long)word) - 1;
                        word &= word - 1ull;
                        const uint4 a = *reinterpret_cast<const uint4 *>(rtq + qb * ldrt32);
                        v.x ^= a.x; v.y ^= a.y; v.z ^= a.z; v.w ^= a.w;
                    }
                }
            }
            *reinterpret_cast<uint4 *>(PT + j * ldpt32 + w0 + q) = v;
        }
        tin[row][q] = v.x;
        tin[row][q + 1] = v.y;
        tin[row][q + 2] = v.z;
        tin[row][q + 3] = v.w;
    }
    __syncthreads();
    transpose_tile_smem(tin, warp, lane);
    __syncthreads();
    const IT ow0 = r0 >> 5;
    // ldp32 is a multiple of 8 and ow0 + q of 4: whole 16-byte words
    if (ow0 + q >= ldp32) return;
#pragma unroll
    for (int k = 0; k < kTW / 4; ++k) {
        const int row = row0 + (kTT / 4) * k;
        const IT orow = c0 + row;
        if (orow >= rows) continue;
        if (IQP_IN((int64_t)orow * ldp32 + ow0 + q + 3, (int64_t)rows * ldp32, 9))
            *reinterpret_cast<uint4 *>(P + orow * ldp32 + ow0 + q) =
                make_uint4(tin[row][q], tin[row][q + 1], tin[row][q + 2], tin[row][q + 3]);
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
    const int64_t nw = (n + 63) >> 6;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *row = G + j * ldg;
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
        if (IQP_IN(j, m, 13)) sup[j] = make_int4(q0, q1, q2, cnt);
    }
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

// Support-gather parities: RT (n x ldpt words) is scratch; writes PT
// (m x ldpt words: bits over rows, zero beyond `rows`) and, if P != nullptr,
// P (rows x ldp words: bits over gates, zero beyond m). With the gates'
// support list `sup` (and ldpt, ldp multiples of 4) P^T and P come from one
// fused pass; without it P^T is gathered, then transposed into P.
cudaError_t launch_parity_gather(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr, const uint64_t *G,
                                 int64_t m, int64_t ldg, uint64_t *P, int64_t ldp, uint64_t *PT, int64_t ldpt,
                                 uint64_t *RT, cudaStream_t st, const int4 *sup) {
    cudaError_t e = bit_transpose(R, rows, n, ldr, RT, ldpt, st);
    if (e != cudaSuccess) return e;
    if (sup != nullptr && P != nullptr && ldpt % 4 == 0 && ldp % 4 == 0) {
        // with the gates' support list (launch_support_list): P^T and P from one pass
        const int64_t gx = cdiv(m, kTT);
        const int64_t gy = cdiv(rows, kTT);
        if (gx * gy > 0x7FFFFFFFll) return cudaErrorInvalidValue;
        // 32-bit element indices where every one of this launch fits
        const int64_t lim = (int64_t)1 << 31;
        const bool i32 = m * 2 * ldpt < lim && rows * 2 * ldp < lim && n * 2 * ldpt < lim && m * ldg < lim &&
                         gx * kTT < lim && gy * kTT < lim;
        LaunchScope ls(IQP_KERNEL_PARITY, st);
        if (i32)
            k_gather_transpose<int32_t><<<(unsigned)(gx * gy), kTT, 0, st>>>(
                sup, G, ldg, n, m, rows, reinterpret_cast<const uint32_t *>(RT), 2 * ldpt,
                reinterpret_cast<uint32_t *>(PT), 2 * ldpt, reinterpret_cast<uint32_t *>(P), 2 * ldp, gx);
        else
            k_gather_transpose<int64_t><<<(unsigned)(gx * gy), kTT, 0, st>>>(
                sup, G, ldg, n, m, rows, reinterpret_cast<const uint32_t *>(RT), 2 * ldpt,
                reinterpret_cast<uint32_t *>(PT), 2 * ldpt, reinterpret_cast<uint32_t *>(P), 2 * ldp, gx);
        return cudaGetLastError();
    }
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
