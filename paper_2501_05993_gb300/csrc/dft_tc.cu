// Batched tone DFT on the tensor cores (tcgen05): T_i = sum_b P[b] e^{-j2 pi ib/N}
// for C channels at once (the "DFT(P)" step of Sec. 2 after the L-to-N fold of
// Eq. 2), as one real contraction
//
//   T (C x 2N, Re T_i and Im T_i side by side) = [Re P | Im P] (C x 2N) . W,
//   W (2N x 2N): column 2i = (cos; sin), column 2i + 1 = (-sin; cos) of the
//   angles 2 pi (i b mod N) / N (rows b < N for Re P, then Im P),
//
// which is dense, so it belongs on the tensor cores.  The operands are split
// into parts of the MMA type whose sum carries FP32's precision: split TF32,
// x = h + l (two 11-bit parts, 2^-22 of x left out) with the products
// h.h + h.l + l.h; split BF16, x = h + m + l (three 8-bit parts, 2^-26 left
// out) with the six products of total order <= 2 (h.h, h.m, m.h, h.l, l.h,
// m.m; the rest are below 2^-24 of the result).
//
// Accumulation.  The tensor cores add an MMA's products into the FP32
// accumulator with about one unit in the last place of error, in the same
// direction every time, so an accumulator that takes every MMA of a long
// contraction drifts by (MMAs) x ulp (measured: 7.6e-6 of max|T| at N = 1024
// for one TF32 accumulator over 256 MMAs).  Here each K chunk (128 bytes of
// K per row: 32 TF32 or 64 BF16 values) starts a fresh accumulator in tensor
// memory, its small cross products first and its h.h products last, and
// eight drain warps move the chunk's sum into FP32 registers (round to
// nearest) while the next chunk accumulates into the other of two TMEM
// buffers.  The drift per chunk is then a few ulps of that chunk's share of
// T, and the chunk sums add like an ordinary FP32 sum.
//
// Kernels.  split_p_kernel writes P as split operand tiles in the shared-
// memory image layout.  dft_tc_kernel: a CTA owns 128 channels (MMA M, rows
// in TMEM lanes) x up to 128 output columns (MMA N) and walks K = 2N chunk
// by chunk; a producer thread streams each chunk's operand and weight parts
// into shared-memory stages with 1-D bulk copies, an MMA thread issues the
// chunk's 4 K-steps x products and commits them to the stage's empty barrier
// and to the TMEM buffer's full barrier, and the drain warps add the buffer
// into registers, release it, and at the end park the tile in shared memory
// from where all threads write complex T row by row.  Shared-memory tiles use
// the no-swizzle K-major layout: 8-row x 16-byte core matrices, the core
// matrices of one 8-row band along K `rows/8 * 128` bytes apart (leading byte
// offset) and consecutive bands 128 bytes apart (stride byte offset).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "internal.cuh"
#include "ptx.cuh"

namespace {

using namespace pcal_ptx;

constexpr int kTcM = 128;                       // channels per tile (MMA M)
constexpr int kTcThreads = 384;                 // 12 warps
constexpr int kDrainWarp0 = 4;                  // warps 4..11 drain the accumulators
constexpr int kDrainWarps = 8;

// Per mode: parts per operand, products per K-step, tile width and pipeline
// depth.  The MMAs read their operands from shared memory, and with
// 128 x 128 tiles those reads plus the copies filling the stages need more
// shared-memory bandwidth than an SM has (split TF32 at its peak: ~109 B per
// clock of operand reads and ~73 B of fills against 128 B), which held the
// tensor pipe near 50-65 %.  Both modes therefore take 128 x 256 tiles (each
// A byte feeds twice the columns).  Split TF32: K chunks of 128 bytes per
// row, two 96 KB stages; split BF16 (three parts): K chunks of 64 bytes, three
// 72 KB stages.  192 / 216 KB of shared memory, one CTA per SM.
template <int MODE>
struct TcCfg {
    static constexpr bool kTf32 = MODE == PCAL_DFT_TC_TF32X3;
    static constexpr int kParts = kTf32 ? 2 : 3;
    static constexpr int kProducts = kTf32 ? 3 : 6;
    static constexpr int kChunk = kTf32 ? 128 : 64;                  // bytes of K per row and chunk
    static constexpr int kATile = kTcM * kChunk;                     // one part of a row tile's chunk
    static constexpr int kImageWords = kATile / 16;                  // 16-byte words of one tile image
    static constexpr int kNT = 256;                                  // output columns per tile
    static constexpr int kBTile = kNT * kChunk;                      // one weight part per chunk
    static constexpr int kStageBytes = kParts * (kATile + kBTile);
    static constexpr int kStages = kTf32 ? 2 : 3;
    static constexpr int kSmem = kStages * kStageBytes;
    static constexpr int kAccCols = kNT;                             // TMEM columns of one accumulator buffer
    static constexpr int kTmemCols = 2 * kAccCols;                   // two buffers (a power of two)
};

// The products of a K-step as (part of A, part of B), the small cross
// products first and h.h last, so that the accumulator is still small while
// most of the MMAs add into it.
__host__ __device__ constexpr int prod_a(int mode, int p) {
    return mode == PCAL_DFT_TC_TF32X3 ? (p == 1 ? 1 : 0) : (p == 0 ? 1 : p == 2 ? 2 : p == 4 ? 1 : 0);
}
__host__ __device__ constexpr int prod_b(int mode, int p) {
    return mode == PCAL_DFT_TC_TF32X3 ? (p == 0 ? 1 : 0) : (p == 0 ? 1 : p == 1 ? 2 : p == 3 ? 1 : 0);
}
// TF32: (0,1) (1,0) (0,0);  BF16: (1,1) (0,2) (2,0) (0,1) (1,0) (0,0)

// Byte offset of element (r, k) of a rows x (128 bytes of K) tile, elements
// of `esize` bytes, in the no-swizzle K-major core-matrix layout.
__host__ __device__ inline uint32_t tile_offset(int r, int k, int rows, int esize) {
    const int kb = k * esize;  // byte position along K
    return (uint32_t)(((kb >> 4) * (rows >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (kb & 15));
}

// Round to TF32 (10 stored mantissa bits), to nearest, ties away from zero,
// as cvt.rna.tf32.f32 does; the result is an FP32 bit pattern.
__host__ __device__ inline uint32_t tf32_bits_rna(float x) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(x);
#else
    memcpy(&u, &x, 4);
#endif
    if ((u & 0x7f800000u) == 0x7f800000u) return u;  // inf, nan: unchanged
    return (u + 0x1000u) & 0xffffe000u;
}

// Round to BF16 (7 stored mantissa bits), to nearest even.
__host__ __device__ inline uint16_t bf16_bits_rn(float x) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(x);
#else
    memcpy(&u, &x, 4);
#endif
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

__host__ __device__ inline float f32_of_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    memcpy(&x, &u, 4);
    return x;
#endif
}

// Split x into the mode's parts (bit patterns in the low bits).  Each
// remainder x - part is exact in FP32: a part is x rounded to fewer bits.
template <int MODE>
__host__ __device__ inline void split_parts(float x, uint32_t* part) {
    if (MODE == PCAL_DFT_TC_TF32X3) {
        part[0] = tf32_bits_rna(x);
        part[1] = tf32_bits_rna(x - f32_of_bits(part[0]));
    } else {
        part[0] = bf16_bits_rn(x);
        const float r1 = x - f32_of_bits(part[0] << 16);
        part[1] = bf16_bits_rn(r1);
        const float r2 = r1 - f32_of_bits(part[1] << 16);
        part[2] = bf16_bits_rn(r2);
    }
}

template <int MODE>
__host__ __device__ constexpr int esize_of() {
    return MODE == PCAL_DFT_TC_TF32X3 ? 4 : 2;
}

// Split x, written at parts[p] + offset for each part p (aligned to the
// element size).
template <int MODE>
__host__ __device__ inline void split_store(float x, uint8_t* const* parts, uint32_t offset) {
    uint32_t v[3];
    split_parts<MODE>(x, v);
    for (int p = 0; p < TcCfg<MODE>::kParts; ++p) {
        if (MODE == PCAL_DFT_TC_TF32X3)
            *reinterpret_cast<uint32_t*>(parts[p] + offset) = v[p];
        else
            *reinterpret_cast<uint16_t*>(parts[p] + offset) = (uint16_t)v[p];
    }
}

// Element W[n][k] of the transposed weight matrix (row n = output column,
// k = contraction index) from the FP64 twiddles tw[m] = e^{-j 2 pi m/N}.
// Output columns interleave the parts of each tone (column 2i = Re T_i,
// 2i + 1 = Im T_i), so a tile's row is a contiguous run of complex T.
inline double weight(const double* twr, const double* twi, int N, int n, int k) {
    const int i = n / 2;                  // tone
    const int b = k < N ? k : k - N;      // residue
    const int m = (int)(((int64_t)i * b) % N);
    const double c = twr[m], s = twi[m];  // e^{-j theta} = c + j s, s = -sin
    if (n % 2 == 0) return k < N ? c : -s;  // Re T = Re P cos + Im P sin
    return k < N ? s : c;                   // Im T = -Re P sin + Im P cos
}

// ---- device side ------------------------------------------------------------

__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
template <int MODE>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if (MODE == PCAL_DFT_TC_TF32X3)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
}
// 32 consecutive TMEM columns of the warp's 32 lanes (one column per
// register), then wait for the load.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: start, leading byte offset (between core
// matrices along K), stride byte offset (between 8-row bands), the fixed
// 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor: FP32 accumulator, A and B of the mode's type, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int MODE>
__device__ __forceinline__ uint32_t instr_desc(int n) {
    const uint32_t ab = MODE == PCAL_DFT_TC_TF32X3 ? 2u : 1u;  // TF32 = 2, BF16 = 1
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

struct DftTcArgs {
    float2* T;         // [C][N]
    int64_t C;
    int N;
    int n_cols;        // 2N rounded up to 16
    int k_chunks;      // chunks of K = 2N
    const uint8_t* a;  // operand tiles of P: [row tile][chunk] x parts x kATile bytes (per mode)
    const uint8_t* w;  // weight tiles: [column tile][chunk] x parts x (tile rows x 128) bytes
    unsigned int* err;
};

// P -> split operand tiles: row tile mt, chunk kc holds rows 128 mt.. and K
// values kc*KC.. of [Re P | Im P] (zeros past C and 2N) as one tile image
// per part.  With 128 rows, 16-byte word w = g*128 + r of an image is row
// r's K values g*V .. g*V+V-1 of the chunk (V = 16 / element size: one core-
// matrix row), so a thread per word reads V consecutive values of one row of
// P (whole sectors) and writes that word of every part.

template <int MODE>
__host__ __device__ inline void split_word(const float2* __restrict__ P, int64_t C, int N, int k_chunks,
                                           int64_t blk, int w, uint4* out) {
    constexpr int ES = esize_of<MODE>();
    constexpr int KC = TcCfg<MODE>::kChunk / ES;
    constexpr int V = 16 / ES;
    constexpr int NP = TcCfg<MODE>::kParts;
    const int r = w % kTcM, g = w / kTcM;
    const int64_t c = (blk / k_chunks) * kTcM + r;
    const int kk0 = (int)(blk % k_chunks) * KC + g * V;
    float x[V];
    for (int j = 0; j < V; ++j) x[j] = 0.f;
    if (c < C) {
        const bool im = kk0 >= N;
        const int64_t src = c * N + (im ? kk0 - N : kk0);
        const bool whole = kk0 + V <= (im ? 2 * N : N);
        if (whole && (reinterpret_cast<uintptr_t>(P + src) & 15) == 0) {
            const float4* q = reinterpret_cast<const float4*>(P + src);
#pragma unroll
            for (int j = 0; j < V / 2; ++j) {
                const float4 v = q[j];
                x[2 * j] = im ? v.y : v.x;
                x[2 * j + 1] = im ? v.w : v.z;
            }
        } else {
            for (int j = 0; j < V; ++j) {
                const int kk = kk0 + j;
                if (kk < N)
                    x[j] = P[c * N + kk].x;
                else if (kk < 2 * N)
                    x[j] = P[c * N + kk - N].y;
            }
        }
    }
    uint32_t word[NP][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if constexpr (MODE == PCAL_DFT_TC_TF32X3) {
            uint32_t v[3];
            split_parts<MODE>(x[i], v);
#pragma unroll
            for (int p = 0; p < NP; ++p) word[p][i] = v[p];
        } else {
            uint32_t v0[3], v1[3];
            split_parts<MODE>(x[2 * i], v0);
            split_parts<MODE>(x[2 * i + 1], v1);
#pragma unroll
            for (int p = 0; p < NP; ++p) word[p][i] = v0[p] | v1[p] << 16;
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) out[p] = make_uint4(word[p][0], word[p][1], word[p][2], word[p][3]);
}

// Word (g*128 + r) of a tile image that thread e of the tile writes.  Split
// BF16: 8 consecutive threads take one row's 8 words (a warp reads 4 rows'
// runs of P), then the next rows; split TF32 (half the values per word)
// keeps one row per thread.
template <int MODE>
__host__ __device__ inline int split_word_of_thread(int e) {
    constexpr int kRowWords = TcCfg<MODE>::kChunk / 16;  // words of one row of a chunk
    return MODE == PCAL_DFT_TC_BF16X6 ? (e % kRowWords) * kTcM + e / kRowWords : e;
}

template <int MODE>
__global__ void __launch_bounds__(256) split_p_kernel(const float2* __restrict__ P, int64_t C, int N, int k_chunks,
                                                      uint4* __restrict__ out, int64_t words) {
    constexpr int NP = TcCfg<MODE>::kParts;
    constexpr int kImageWords = TcCfg<MODE>::kImageWords;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
        const int64_t blk = i / kImageWords;
        const int w = split_word_of_thread<MODE>((int)(i % kImageWords));
        uint4 part[NP];
        split_word<MODE>(P, C, N, k_chunks, blk, w, part);
#pragma unroll
        for (int p = 0; p < NP; ++p) out[(blk * NP + p) * kImageWords + w] = part[p];
    }
}


// One CTA: 128 channels x up to 128 output columns.  Thread 0 streams the
// operand and weight parts of each chunk through kStages shared-memory stages
// (bulk copies, full barriers); thread 32 waits for a stage and for the TMEM
// buffer of the chunk (kc % 2) to be drained, issues the chunk's MMAs into
// that buffer (the first one overwrites it) and commits them to the stage's
// empty barrier and the buffer's full barrier; warps 4..11 add each drained
// buffer into FP32 registers (warp w: TMEM lanes 32 (w % 4) .., columns
// 64 ((w - 4) / 4) ..) and release it.
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) dft_tc_kernel(const DftTcArgs a) {
    using Cfg = TcCfg<MODE>;
    constexpr int ES = esize_of<MODE>();
    constexpr int kATile = Cfg::kATile;
    constexpr int KC = Cfg::kChunk / ES;  // K values per chunk
    constexpr int KS = 32 / ES;           // K values per MMA
    constexpr int NP = Cfg::kParts, kStages = Cfg::kStages, kStageBytes = Cfg::kStageBytes;
    constexpr int kAccCols = Cfg::kAccCols, kTmemCols = Cfg::kTmemCols;
    constexpr int kDrainCols = kAccCols / 2;  // columns per drain warp
    constexpr int kPieces = kDrainCols / 32;  // 32-column TMEM loads per drain warp
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t mt = blockIdx.x;
    const int64_t m0 = mt * kTcM;
    const int n0 = blockIdx.y * Cfg::kNT;
    const int nt = a.n_cols - n0 < Cfg::kNT ? a.n_cols - n0 : Cfg::kNT;  // a multiple of 16
    const uint32_t w_bytes = (uint32_t)nt * Cfg::kChunk;                 // one weight part of a chunk
    if (warp == 2) {
        tc_alloc(&s_tmem, kTmemCols);
        tc_relinquish();
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kDrainWarps);
        }
        mbar_init(&done, 1);
        s_fail = 0;
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        // ---- producer ----
        const uint8_t* atile = a.a + (size_t)mt * a.k_chunks * NP * kATile;
        const uint8_t* wtile = a.w + (size_t)blockIdx.y * a.k_chunks * NP * Cfg::kBTile;
        int issued = 0;
        for (int kc = 0; kc < a.k_chunks; ++kc) {
            const int s = kc % kStages;
            if (kc >= kStages && !mbar_wait(&empty[s], (uint32_t)((kc / kStages - 1) & 1))) {
                atomicOr(a.err, PCAL_DERR_EMPTY_WAIT);
                s_fail = 1;
                break;
            }
            issued = kc + 1;
            uint8_t* st = smem + (size_t)s * kStageBytes;
            mbar_arrive_expect_tx(&full[s], NP * kATile + NP * w_bytes);
            bulk_load(st, atile + (size_t)kc * NP * kATile, NP * kATile, &full[s]);
            bulk_load(st + NP * kATile, wtile + (size_t)kc * NP * Cfg::kBTile, NP * w_bytes, &full[s]);
        }
        if (s_fail) {
            // copies in flight must land before the CTA's shared memory is reused
            for (int kc = issued - kStages > 0 ? issued - kStages : 0; kc < issued; ++kc)
                if (!mbar_wait(&full[kc % kStages], (uint32_t)((kc / kStages) & 1))) atomicOr(a.err, PCAL_DERR_DRAIN_WAIT);
        }
    } else if (tid == 32) {
        // ---- MMA issuer ----
        const uint32_t idesc = instr_desc<MODE>(nt);
        const uint32_t lbo_a = (kTcM / 8) * 128, lbo_b = (uint32_t)(nt / 8) * 128;
        bool ok = true;
        for (int kc = 0; kc < a.k_chunks; ++kc) {
            const int s = kc % kStages, b = kc & 1;
            if (!mbar_wait(&full[s], (uint32_t)((kc / kStages) & 1))) {
                atomicOr(a.err, PCAL_DERR_FULL_WAIT);
                ok = false;
            } else if (kc >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)(((kc >> 1) - 1) & 1))) {
                atomicOr(a.err, PCAL_DERR_FULL_WAIT);
                ok = false;
            }
            if (!ok) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t st = smem_addr(smem + (size_t)s * kStageBytes);
            const uint32_t d = tmem + (uint32_t)(b * kAccCols);
            uint32_t accumulate = 0u;  // the chunk's first MMA overwrites the buffer
#pragma unroll
            for (int p = 0; p < Cfg::kProducts; ++p) {
                const uint32_t pa = st + (uint32_t)(prod_a(MODE, p) * kATile);
                const uint32_t pb = st + (uint32_t)(NP * kATile) + (uint32_t)prod_b(MODE, p) * w_bytes;
#pragma unroll
                for (int k = 0; k < KC / KS; ++k) {
                    const uint64_t ad = smem_desc(pa + (uint32_t)k * 2 * lbo_a, lbo_a, 128);
                    const uint64_t bd = smem_desc(pb + (uint32_t)k * 2 * lbo_b, lbo_b, 128);
                    tc_mma<MODE>(d, ad, bd, idesc, accumulate);
                    accumulate = 1u;
                }
            }
            tc_commit(&empty[s]);     // the stage is free once these MMAs are done
            tc_commit(&acc_full[b]);  // and the buffer holds the chunk's sum
        }
        if (ok) tc_commit(&done);
    } else if (warp >= kDrainWarp0) {
        // ---- drain warps ----
        const int q = warp & 3;                                   // TMEM lane quadrant of this warp
        const int c0 = ((warp - kDrainWarp0) >> 2) * kDrainCols;  // first column of this warp
        const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
        const int pieces = nt > c0 ? (nt - c0 >= kDrainCols ? kPieces : (nt - c0 + 31) / 32) : 0;  // 32-column loads
        float sum[kDrainCols];
#pragma unroll
        for (int j = 0; j < kDrainCols; ++j) sum[j] = 0.f;
        bool ok = true;
        for (int kc = 0; kc < a.k_chunks; ++kc) {
            const int b = kc & 1;
            if (!mbar_wait(&acc_full[b], (uint32_t)((kc >> 1) & 1))) {
                atomicOr(a.err, PCAL_DERR_DRAIN_WAIT);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t base = tmem + lane_addr + (uint32_t)(b * kAccCols + c0);
            uint32_t v[32];
#pragma unroll
            for (int pc = 0; pc < kPieces; ++pc) {
                if (pc < pieces) {
                    tc_ld32(base + 32u * pc, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) sum[32 * pc + j] += __uint_as_float(v[j]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (!ok) {
            s_fail = 1;
        } else {
            // every MMA has completed (the last buffer's commit covers them all)
            // and every copy has landed: the stages are free.  Park the rows
            // (stride 129 floats: no bank conflicts).
            constexpr int kRow = Cfg::kNT + 1;
            float* sT = reinterpret_cast<float*>(smem);
            const int r = 32 * q + lane;
#pragma unroll
            for (int j = 0; j < kDrainCols; ++j)
                if (c0 + j < nt) sT[r * kRow + c0 + j] = sum[j];
        }
    }
    // every thread: wait for the last MMAs (the issuer committed `done`)
    __syncthreads();
    const bool have = __syncthreads_and(!s_fail && mbar_wait(&done, 0)) != 0;  // uniform over the CTA
    if (!have && tid == 0) atomicOr(a.err, PCAL_DERR_DRAIN_WAIT);
    tc_fence_after();
    if (have) {
        // all threads write the tile's rows of complex T, consecutive threads
        // on consecutive tones
        constexpr int kRow = Cfg::kNT + 1;
        const float* sT = reinterpret_cast<const float*>(smem);
        const int tones = nt / 2, t0 = n0 / 2;
        for (int e = tid; e < kTcM * tones; e += kTcThreads) {
            const int rr = e / tones, i = e % tones;
            const int64_t c = m0 + rr;
            if (c < a.C && t0 + i < a.N)
                a.T[c * a.N + t0 + i] = make_float2(sT[rr * kRow + 2 * i], sT[rr * kRow + 2 * i + 1]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        tc_dealloc(tmem, kTmemCols);
    }
}

// FP32 CUDA-core reference mode: one block per channel, the N tones from P in
// shared memory with the twiddles of the table (FP32 sums).
__global__ void dft_fp32_kernel(const float2* __restrict__ P, float2* __restrict__ T, int N,
                                const float2* __restrict__ tw) {
    extern __shared__ float2 sp[];
    const int64_t c = blockIdx.x;
    for (int b = threadIdx.x; b < N; b += blockDim.x) {
        sp[b] = P[c * N + b];
        sp[N + b] = tw[b];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        float re = 0.f, im = 0.f;
        int m = 0;
        for (int b = 0; b < N; ++b) {
            const float2 p = sp[b], w = sp[N + m];
            re = fmaf(p.x, w.x, fmaf(-p.y, w.y, re));
            im = fmaf(p.x, w.y, fmaf(p.y, w.x, im));
            m += i;
            if (m >= N) m -= N;
        }
        T[c * N + i] = make_float2(re, im);
    }
}

}  // namespace

struct pcal_dft {
    int N, mode, n_cols, k_chunks, col_tiles, parts;
    uint8_t* d_w;     // weight tiles (tensor-core modes)
    uint8_t* d_a;     // operand tiles of P (workspace)
    size_t a_cap;     // bytes of d_a
    float2* d_tw;     // FP32 twiddles (CUDA-core mode)
    unsigned int* d_err;
};

namespace {

// output columns per tile of a tensor-core mode
inline int tile_cols(int mode) {
    return mode == PCAL_DFT_TC_TF32X3 ? TcCfg<PCAL_DFT_TC_TF32X3>::kNT : TcCfg<PCAL_DFT_TC_BF16X6>::kNT;
}

inline int parts_of(int mode) {
    return mode == PCAL_DFT_TC_TF32X3 ? TcCfg<PCAL_DFT_TC_TF32X3>::kParts : TcCfg<PCAL_DFT_TC_BF16X6>::kParts;
}

// bytes of K per row and chunk of a tensor-core mode
inline int chunk_bytes(int mode) {
    return mode == PCAL_DFT_TC_TF32X3 ? TcCfg<PCAL_DFT_TC_TF32X3>::kChunk : TcCfg<PCAL_DFT_TC_BF16X6>::kChunk;
}

// Weight tile of column tile t, chunk kc, in the shared-memory image the
// kernel copies (rows = the tile's columns, the mode's chunk of K per row): part p
// at out + p * part_stride.  Returns the tile's rows.
int build_weight_tile(int N, int mode, int t, int kc, const double* twr, const double* twi, uint8_t* out,
                      size_t part_stride) {
    const int n_cols = (2 * N + 15) / 16 * 16;
    const int tc = tile_cols(mode);
    const int n0 = t * tc;
    const int nt = n_cols - n0 < tc ? n_cols - n0 : tc;
    const int es = mode == PCAL_DFT_TC_TF32X3 ? 4 : 2;
    const int kcv = chunk_bytes(mode) / es;
    const int np = parts_of(mode);
    uint8_t* parts[3] = {out, out + part_stride, out + 2 * part_stride};
    for (int p = 0; p < np; ++p) memset(parts[p], 0, (size_t)nt * chunk_bytes(mode));
    for (int r = 0; r < nt; ++r) {
        const int n = n0 + r;
        for (int k = 0; k < kcv; ++k) {
            const int kk = kc * kcv + k;
            const float x = (n < 2 * N && kk < 2 * N) ? (float)weight(twr, twi, N, n, kk) : 0.f;
            const uint32_t o = tile_offset(r, k, nt, es);
            if (mode == PCAL_DFT_TC_TF32X3)
                split_store<PCAL_DFT_TC_TF32X3>(x, parts, o);
            else
                split_store<PCAL_DFT_TC_BF16X6>(x, parts, o);
        }
    }
    return nt;
}

void twiddles(int N, double* twr, double* twi) {
    for (int m = 0; m < N; ++m) {
        // e^{-j 2 pi m/N} from the exactly reduced angle
        const double th = 2.0 * M_PI * (double)m / (double)N;
        twr[m] = cos(th);
        twi[m] = -sin(th);
    }
}

}  // namespace

extern "C" int pcal_dft_weights_host(int N, int mode, int tile, int chunk, void* parts, int* rows, int* n_parts) {
    if (N < 1 || N > PCAL_BATCH_MAX_N || !parts || !rows || !n_parts) return PCAL_EINVAL;
    if (mode != PCAL_DFT_TC_TF32X3 && mode != PCAL_DFT_TC_BF16X6) return PCAL_EINVAL;
    const int n_cols = (2 * N + 15) / 16 * 16;
    const int es = mode == PCAL_DFT_TC_TF32X3 ? 4 : 2;
    const int kcv = chunk_bytes(mode) / es;
    const int k_chunks = (2 * N + kcv - 1) / kcv;
    if (tile < 0 || tile * tile_cols(mode) >= n_cols || chunk < 0 || chunk >= k_chunks) return PCAL_EINVAL;
    double* tw = new (std::nothrow) double[2 * (size_t)N];
    if (!tw) return PCAL_ENOMEM;
    twiddles(N, tw, tw + N);
    *rows = build_weight_tile(N, mode, tile, chunk, tw, tw + N, static_cast<uint8_t*>(parts),
                              (size_t)tile_cols(mode) * chunk_bytes(mode));
    *n_parts = parts_of(mode);
    delete[] tw;
    return PCAL_OK;
}

extern "C" int pcal_dft_create(int N, int mode, pcal_dft** out) {
    if (!out || N < 1 || N > PCAL_BATCH_MAX_N) return PCAL_EINVAL;
    if (mode != PCAL_DFT_FP32 && mode != PCAL_DFT_TC_TF32X3 && mode != PCAL_DFT_TC_BF16X6) return PCAL_EINVAL;
    pcal_dft* d = new (std::nothrow) pcal_dft();
    if (!d) return PCAL_ENOMEM;
    memset(static_cast<void*>(d), 0, sizeof(*d));
    d->N = N;
    d->mode = mode;
    d->n_cols = (2 * N + 15) / 16 * 16;
    const int tc = mode == PCAL_DFT_FP32 ? 0 : tile_cols(mode);
    d->col_tiles = mode == PCAL_DFT_FP32 ? 0 : (d->n_cols + tc - 1) / tc;
    d->parts = mode == PCAL_DFT_FP32 ? 0 : parts_of(mode);
    const int es = mode == PCAL_DFT_TC_TF32X3 ? 4 : 2;
    const int cb = mode == PCAL_DFT_FP32 ? 128 : chunk_bytes(mode);
    d->k_chunks = (2 * N + cb / es - 1) / (cb / es);
    double* tw = new (std::nothrow) double[2 * (size_t)N];
    if (!tw) {
        delete d;
        return PCAL_ENOMEM;
    }
    twiddles(N, tw, tw + N);
    cudaError_t e = cudaMalloc(&d->d_err, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(d->d_err, 0, sizeof(unsigned int));
    if (e == cudaSuccess && mode == PCAL_DFT_FP32) {
        float2* h = new (std::nothrow) float2[N];
        if (!h) e = cudaErrorMemoryAllocation;
        for (int m = 0; h && m < N; ++m) h[m] = make_float2((float)tw[m], (float)tw[N + m]);
        if (e == cudaSuccess) e = cudaMalloc(&d->d_tw, N * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemcpy(d->d_tw, h, N * sizeof(float2), cudaMemcpyHostToDevice);
        delete[] h;
    } else if (e == cudaSuccess) {
        // per (column tile, chunk): the parts of the tile's rows, one after the
        // other (a ragged last tile keeps its rows together): one copy per chunk
        const size_t block = (size_t)d->parts * tc * cb;
        const size_t bytes = (size_t)d->col_tiles * d->k_chunks * block;
        uint8_t* h = new (std::nothrow) uint8_t[bytes];
        if (!h) e = cudaErrorMemoryAllocation;
        for (int t = 0; h && t < d->col_tiles; ++t) {
            const int nt = d->n_cols - t * tc < tc ? d->n_cols - t * tc : tc;
            for (int kc = 0; kc < d->k_chunks; ++kc)
                build_weight_tile(N, mode, t, kc, tw, tw + N, h + ((size_t)t * d->k_chunks + kc) * block,
                                  (size_t)nt * cb);
        }
        if (e == cudaSuccess) e = cudaMalloc(&d->d_w, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(d->d_w, h, bytes, cudaMemcpyHostToDevice);
        delete[] h;
    }
    delete[] tw;
    if (e == cudaSuccess && mode != PCAL_DFT_FP32) {
        e = mode == PCAL_DFT_TC_TF32X3
                ? cudaFuncSetAttribute(dft_tc_kernel<PCAL_DFT_TC_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TcCfg<PCAL_DFT_TC_TF32X3>::kSmem)
                : cudaFuncSetAttribute(dft_tc_kernel<PCAL_DFT_TC_BF16X6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TcCfg<PCAL_DFT_TC_BF16X6>::kSmem);
    }
    if (e != cudaSuccess) {
        pcal_dft_destroy(d);
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PCAL_ENOMEM : PCAL_ECUDA;
    }
    *out = d;
    return PCAL_OK;
}

extern "C" int pcal_dft_destroy(pcal_dft* d) {
    if (!d) return PCAL_OK;
    cudaDeviceSynchronize();
    cudaFree(d->d_w);
    cudaFree(d->d_a);
    cudaFree(d->d_tw);
    cudaFree(d->d_err);
    delete d;
    return PCAL_OK;
}

// Operand workspace for C channels (allocates: not under stream capture).
cudaError_t dft_reserve(pcal_dft* d, int64_t C) {
    if (d->mode == PCAL_DFT_FP32 || C <= 0) return cudaSuccess;
    const size_t need = (size_t)((C + kTcM - 1) / kTcM) * d->k_chunks * d->parts * kTcM * chunk_bytes(d->mode);
    if (need <= d->a_cap) return cudaSuccess;
    cudaFree(d->d_a);
    d->d_a = nullptr;
    d->a_cap = 0;
    const cudaError_t e = cudaMalloc(&d->d_a, need);
    if (e == cudaSuccess) d->a_cap = need;
    return e;
}

cudaError_t launch_dft(pcal_dft* d, const float2* P, int64_t C, float2* T, cudaStream_t s, unsigned int* err) {
    if (C <= 0) return cudaSuccess;
    if (d->mode == PCAL_DFT_FP32) {
        dft_fp32_kernel<<<(unsigned)C, 256, 2 * d->N * sizeof(float2), s>>>(P, T, d->N, d->d_tw);
        return cudaGetLastError();
    }
    const int64_t m_tiles = (C + kTcM - 1) / kTcM;
    const size_t a_tile = (size_t)kTcM * chunk_bytes(d->mode);  // one part of a row tile's chunk
    if ((size_t)m_tiles * d->k_chunks * d->parts * a_tile > d->a_cap) return cudaErrorInvalidValue;  // dft_reserve first
    const int64_t words = m_tiles * d->k_chunks * (int64_t)(a_tile / 16);  // one thread per word (all parts)
    const int64_t blocks = (words + 255) / 256;
    const int sgrid = (int)(blocks < 32 * 152 ? blocks : 32 * 152);
    uint4* a_words = reinterpret_cast<uint4*>(d->d_a);
    if (d->mode == PCAL_DFT_TC_TF32X3)
        split_p_kernel<PCAL_DFT_TC_TF32X3><<<sgrid, 256, 0, s>>>(P, C, d->N, d->k_chunks, a_words, words);
    else
        split_p_kernel<PCAL_DFT_TC_BF16X6><<<sgrid, 256, 0, s>>>(P, C, d->N, d->k_chunks, a_words, words);
    DftTcArgs a{};
    a.T = T;
    a.a = d->d_a;
    a.C = C;
    a.N = d->N;
    a.n_cols = d->n_cols;
    a.k_chunks = d->k_chunks;
    a.w = d->d_w;
    a.err = err ? err : d->d_err;
    const dim3 grid((unsigned)m_tiles, (unsigned)d->col_tiles);
    if (d->mode == PCAL_DFT_TC_TF32X3)
        dft_tc_kernel<PCAL_DFT_TC_TF32X3><<<grid, kTcThreads, TcCfg<PCAL_DFT_TC_TF32X3>::kSmem, s>>>(a);
    else
        dft_tc_kernel<PCAL_DFT_TC_BF16X6><<<grid, kTcThreads, TcCfg<PCAL_DFT_TC_BF16X6>::kSmem, s>>>(a);
    return cudaGetLastError();
}

extern "C" int pcal_dft_execute(pcal_dft* d, const void* P, int64_t C, void* T, void* stream) {
    if (!d || C < 0 || (C > 0 && (!P || !T))) return PCAL_EINVAL;
    if (C > (int64_t)65535 * kTcM) return PCAL_ETOOLARGE;
    if (dft_reserve(d, C) != cudaSuccess) {
        (void)cudaGetLastError();
        return PCAL_ENOMEM;
    }
    const cudaError_t e = launch_dft(d, static_cast<const float2*>(P), C, static_cast<float2*>(T),
                                     static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PCAL_OK : PCAL_ECUDA;
}

extern "C" int pcal_dft_check(pcal_dft* d, unsigned int* flags_out) {
    if (!d || !flags_out) return PCAL_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(flags_out, d->d_err, sizeof(unsigned int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PCAL_ECUDA;
    return *flags_out ? PCAL_ETIMEOUT : PCAL_OK;
}
