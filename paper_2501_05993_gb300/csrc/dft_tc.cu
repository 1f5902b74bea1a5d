// Batched tone DFT on the tensor cores (tcgen05): T_i = sum_b P[b] e^{-j2 pi ib/N}
// for C channels at once (the "DFT(P)" step of Sec. 2 after the L-to-N fold of
// Eq. 2), as one real contraction
//
//   T (C x 2N, Re T_i and Im T_i side by side) = [Re P | Im P] (C x 2N) . W,
//   W (2N x 2N): column 2i = (cos; sin), column 2i + 1 = (-sin; cos) of the
//   angles 2 pi (i b mod N) / N (rows b < N for Re P, then Im P),
//
// which is dense, so it belongs on the tensor cores.  The operands are split
// in two parts of the MMA type (x = hi + lo, hi = round(x), lo = round(x - hi))
// and three products hi.hi + hi.lo + lo.hi accumulate in FP32 in tensor
// memory.  The tensor cores' FP32 accumulation loses about one unit in the
// last place per MMA, in the same direction, so the error grows with the
// number of MMAs an accumulator takes: the hi.hi products and the small cross
// products go to separate accumulators (split TF32, with twice the MMAs per K,
// also splits hi.hi over even and odd K chunks), added in FP32 at the end
// (error figures: pcal.h).
//
// Kernels.  split_p_kernel writes P as split operand tiles in the shared-
// memory image layout.  dft_tc_kernel: a CTA owns 128 channels (MMA M, rows
// in TMEM lanes) x up to 256 (split BF16) or 128 (split TF32) output columns
// (MMA N) and walks K = 2N in chunks of 128 bytes per row (64 BF16 or 32 TF32
// values); a producer thread streams each chunk's operand and weight tiles
// into shared-memory stages with 1-D bulk copies, an MMA thread issues 4
// K-steps x 3 products per chunk and commits them to the stage's empty
// barrier, and the epilogue parks the accumulators in shared memory and
// writes complex T row by row.  Shared-memory tiles use the no-swizzle
// K-major layout: 8-row x 16-byte core matrices, the core matrices of one
// 8-row band along K `rows/8 * 128` bytes apart (leading byte offset) and
// consecutive bands 128 bytes apart (stride byte offset).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "internal.cuh"
#include "ptx.cuh"

namespace {

using namespace pcal_ptx;

constexpr int kTcM = 128;              // channels per tile (MMA M)
// Output columns per tile (MMA N), stages and accumulators per mode: split
// BF16 (16 K values per MMA) takes 256-column tiles with two accumulators
// (hi.hi, cross products) in 2 stages of 96 KB; split TF32 (8 K values per
// MMA, twice the MMAs per accumulator) 128-column tiles with the hi.hi
// products over even and odd chunks in separate accumulators, in 3 stages
// of 64 KB.
template <int MODE>
struct TcCfg {
    static constexpr bool kWide = MODE == PCAL_DFT_TC_BF16X3;
    static constexpr int kNT = kWide ? 256 : 128;
    static constexpr int kStages = kWide ? 2 : 3;
    static constexpr int kBTile = kNT * 128;                     // bytes of one weight part per chunk
    static constexpr int kStageBytes = 2 * 128 * 128 + 2 * kBTile;  // A hi, A lo, B hi, B lo
    static constexpr int kSmem = kStages * kStageBytes;          // 192 KB either way: one CTA per SM
};
constexpr int kTcThreads = 256;        // 8 warps
constexpr int kChunkBytes = 128;       // bytes of K per row and chunk
constexpr int kATile = kTcM * kChunkBytes;      // 16 KB
constexpr int kTmemCols = 512;                  // the accumulators of either mode (a power of two)

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

// Split x into two parts of the MMA type (bit patterns in the low bits).
template <int MODE>
__host__ __device__ inline void split_parts(float x, uint32_t& h, uint32_t& l) {
    if (MODE == PCAL_DFT_TC_TF32X3) {
        h = tf32_bits_rna(x);
        l = tf32_bits_rna(x - f32_of_bits(h));
    } else {
        h = bf16_bits_rn(x);
        l = bf16_bits_rn(x - f32_of_bits(h << 16));
    }
}

// Split x, written at `hi` and `lo` (aligned to the element size).
template <int MODE>
__host__ __device__ inline void split_store(float x, uint8_t* hi, uint8_t* lo) {
    uint32_t h, l;
    split_parts<MODE>(x, h, l);
    if (MODE == PCAL_DFT_TC_TF32X3) {
        *reinterpret_cast<uint32_t*>(hi) = h;
        *reinterpret_cast<uint32_t*>(lo) = l;
    } else {
        *reinterpret_cast<uint16_t*>(hi) = (uint16_t)h;
        *reinterpret_cast<uint16_t*>(lo) = (uint16_t)l;
    }
}

template <int MODE>
__host__ __device__ constexpr int esize_of() {
    return MODE == PCAL_DFT_TC_TF32X3 ? 4 : 2;
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
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float* v) {
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4);
    v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6);
    v[7] = __uint_as_float(r7);
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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
    const uint8_t* a;  // operand tiles of P: [row tile][chunk] x (hi, lo) x kATile bytes
    const uint8_t* w;  // weight tiles: [column tile][chunk] x 2 kBTile bytes: hi rows, then lo rows
    unsigned int* err;
};

// P -> split operand tiles: row tile mt, chunk kc holds rows 128 mt.. and K
// values kc*KC.. of [Re P | Im P] (zeros past C and 2N) as hi and lo tile
// images.  With 128 rows, 16-byte word w = g*128 + r of an image is row r's
// K values g*V .. g*V+V-1 of the chunk (V = 16 / element size: one core-
// matrix row), so a thread per word reads V consecutive values of one row of
// P (whole sectors) and writes its hi and lo words.
constexpr int kImageWords = kATile / 16;  // 16-byte words of one tile image

template <int MODE>
__host__ __device__ inline void split_word(const float2* __restrict__ P, int64_t C, int N, int k_chunks,
                                           int64_t blk, int w, uint4& hi, uint4& lo) {
    constexpr int ES = esize_of<MODE>();
    constexpr int KC = kChunkBytes / ES;
    constexpr int V = 16 / ES;
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
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if constexpr (MODE == PCAL_DFT_TC_TF32X3) {
            split_parts<MODE>(x[i], h[i], l[i]);
        } else {
            uint32_t h0, l0, h1, l1;
            split_parts<MODE>(x[2 * i], h0, l0);
            split_parts<MODE>(x[2 * i + 1], h1, l1);
            h[i] = h0 | h1 << 16;
            l[i] = l0 | l1 << 16;
        }
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Word (g*128 + r) of a tile image that thread e of the tile writes.  Split
// BF16: 8 consecutive threads take one row's 8 words (a warp reads 4 rows'
// runs of P), then the next rows (18.0 against 19.3 us per launch at
// 4096 x 1024); split TF32 (half the values per word) keeps one row per
// thread (20.0 against 22.8 us).
template <int MODE>
__host__ __device__ inline int split_word_of_thread(int e) {
    constexpr int kRowWords = kChunkBytes / 16;  // words of one row of a chunk
    return MODE == PCAL_DFT_TC_BF16X3 ? (e % kRowWords) * kTcM + e / kRowWords : e;
}

template <int MODE>
__global__ void __launch_bounds__(256) split_p_kernel(const float2* __restrict__ P, int64_t C, int N, int k_chunks,
                                                      uint4* __restrict__ out, int64_t words) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
        const int64_t blk = i / kImageWords;
        const int w = split_word_of_thread<MODE>((int)(i % kImageWords));
        uint4 hi, lo;
        split_word<MODE>(P, C, N, k_chunks, blk, w, hi, lo);
        out[blk * 2 * kImageWords + w] = hi;
        out[blk * 2 * kImageWords + kImageWords + w] = lo;
    }
}


// One CTA: 128 channels x up to TcCfg::kNT output columns.  Thread 0 streams the A
// and B tile pairs of each chunk through kStages shared-memory stages (bulk
// copies, full barriers); thread 32 issues the chunk's 4 K-steps x 3 products
// and commits them to the stage's empty barrier, so a stage is refilled as
// soon as the MMAs that read it are done; a last commit signals the epilogue.
template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) dft_tc_kernel(const DftTcArgs a) {
    constexpr int ES = esize_of<MODE>();
    constexpr int KC = kChunkBytes / ES;  // K values per chunk
    constexpr int KS = 32 / ES;           // K values per MMA
    using Cfg = TcCfg<MODE>;
    constexpr int kTcNMax = Cfg::kNT, kStages = Cfg::kStages, kBTile = Cfg::kBTile, kStageBytes = Cfg::kStageBytes;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t mt = blockIdx.x;
    const int64_t m0 = mt * kTcM;
    const int n0 = blockIdx.y * kTcNMax;
    const int nt = a.n_cols - n0 < kTcNMax ? a.n_cols - n0 : kTcNMax;  // a multiple of 16
    const uint32_t w_bytes = (uint32_t)nt * kChunkBytes;
    if (warp == 0) {
        tc_alloc(&s_tmem, kTmemCols);
        tc_relinquish();
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
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
        const uint8_t* atile = a.a + (size_t)mt * a.k_chunks * 2 * kATile;
        const uint8_t* wtile = a.w + (size_t)blockIdx.y * a.k_chunks * 2 * kBTile;
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
            mbar_arrive_expect_tx(&full[s], 2 * kATile + 2 * w_bytes);
            bulk_load(st, atile + (size_t)kc * 2 * kATile, 2 * kATile, &full[s]);
            bulk_load(st + 2 * kATile, wtile + (size_t)kc * 2 * kBTile, 2 * w_bytes, &full[s]);  // hi and lo
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
            const int s = kc % kStages;
            if (!mbar_wait(&full[s], (uint32_t)((kc / kStages) & 1))) {
                atomicOr(a.err, PCAL_DERR_FULL_WAIT);
                s_fail = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t st = smem_addr(smem + (size_t)s * kStageBytes);
            const uint32_t a_hi = st, a_lo = st + kATile, b_hi = st + 2 * kATile, b_lo = b_hi + w_bytes;
            // hi.hi: one accumulator (wide tiles) or even / odd chunks; cross
            // products: the last accumulator
            const uint32_t d_hh = tmem + (Cfg::kWide ? 0u : (uint32_t)(kc & 1) * kTcNMax);
            const uint32_t d_x = tmem + (Cfg::kWide ? 1u : 2u) * kTcNMax;
            const bool hh_first = Cfg::kWide ? kc == 0 : kc < 2;
#pragma unroll
            for (int k = 0; k < KC / KS; ++k) {
                const uint32_t oa = (uint32_t)k * 2 * lbo_a, ob = (uint32_t)k * 2 * lbo_b;
                const uint64_t ah = smem_desc(a_hi + oa, lbo_a, 128), al = smem_desc(a_lo + oa, lbo_a, 128);
                const uint64_t bh = smem_desc(b_hi + ob, lbo_b, 128), bl = smem_desc(b_lo + ob, lbo_b, 128);
                tc_mma<MODE>(d_hh, ah, bh, idesc, (hh_first && k == 0) ? 0u : 1u);
                tc_mma<MODE>(d_x, ah, bl, idesc, (kc == 0 && k == 0) ? 0u : 1u);
                tc_mma<MODE>(d_x, al, bh, idesc, 1u);
            }
            tc_commit(&empty[s]);  // the stage is free once these MMAs are done
        }
        if (ok) tc_commit(&done);
    }
    // every thread: wait for the last MMAs (the issuer committed `done`)
    __syncthreads();
    const bool have = __syncthreads_and(!s_fail && mbar_wait(&done, 0)) != 0;  // uniform over the CTA
    if (!have && tid == 0) atomicOr(a.err, PCAL_DERR_DRAIN_WAIT);
    tc_fence_after();
    if (have) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows), column half
        // w / 4, adds the three accumulators and parks the rows in shared
        // memory (the stages are free; row stride 129 floats: no bank
        // conflicts), then all threads write the tile's rows of complex T,
        // consecutive threads on consecutive tones.
        constexpr int kRow = kTcNMax + 1;
        float* sT = reinterpret_cast<float*>(smem);
        const int q = warp & 3, half = warp >> 2;
        const int r = 32 * q + (tid & 31);
        const uint32_t lane = (uint32_t)(32 * q) << 16;
        for (int j0 = half * (kTcNMax / 2); j0 < nt && j0 < (half + 1) * (kTcNMax / 2); j0 += 8) {
            float v[8], w[8], x[8];
            tc_ld8(tmem + lane + (uint32_t)j0, v);
            tc_ld8(tmem + lane + (uint32_t)((Cfg::kWide ? 1 : 2) * kTcNMax + j0), x);
            if (!Cfg::kWide && a.k_chunks > 1) {
                tc_ld8(tmem + lane + (uint32_t)(kTcNMax + j0), w);
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] += w[u];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) sT[r * kRow + j0 + u] = v[u] + x[u];
        }
        __syncthreads();
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
    if (warp == 0) {
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
    int N, mode, n_cols, k_chunks, col_tiles;
    uint8_t* d_w;     // weight tiles (tensor-core modes)
    uint8_t* d_a;     // operand tiles of P (workspace)
    size_t a_cap;     // bytes of d_a
    float2* d_tw;     // FP32 twiddles (CUDA-core mode)
    unsigned int* d_err;
};

namespace {

// Weight tiles of column tile t, chunk kc, in the shared-memory image the
// kernel copies (rows = the tile's columns, 128 bytes of K per row).
inline int tile_cols(int mode) {
    return mode == PCAL_DFT_TC_TF32X3 ? TcCfg<PCAL_DFT_TC_TF32X3>::kNT : TcCfg<PCAL_DFT_TC_BF16X3>::kNT;
}

int build_weight_tile(int N, int mode, int t, int kc, const double* twr, const double* twi, uint8_t* hi,
                      uint8_t* lo) {
    const int n_cols = (2 * N + 15) / 16 * 16;
    const int NT = tile_cols(mode);
    const int n0 = t * NT;
    const int nt = n_cols - n0 < NT ? n_cols - n0 : NT;
    const int es = mode == PCAL_DFT_TC_TF32X3 ? 4 : 2;
    const int kcv = kChunkBytes / es;
    memset(hi, 0, (size_t)nt * kChunkBytes);
    memset(lo, 0, (size_t)nt * kChunkBytes);
    for (int r = 0; r < nt; ++r) {
        const int n = n0 + r;
        for (int k = 0; k < kcv; ++k) {
            const int kk = kc * kcv + k;
            const float x = (n < 2 * N && kk < 2 * N) ? (float)weight(twr, twi, N, n, kk) : 0.f;
            const uint32_t o = tile_offset(r, k, nt, es);
            if (mode == PCAL_DFT_TC_TF32X3)
                split_store<PCAL_DFT_TC_TF32X3>(x, hi + o, lo + o);
            else
                split_store<PCAL_DFT_TC_BF16X3>(x, hi + o, lo + o);
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

extern "C" int pcal_dft_weights_host(int N, int mode, int tile, int chunk, void* hi, void* lo, int* rows) {
    if (N < 1 || N > PCAL_BATCH_MAX_N || !hi || !lo || !rows) return PCAL_EINVAL;
    if (mode != PCAL_DFT_TC_TF32X3 && mode != PCAL_DFT_TC_BF16X3) return PCAL_EINVAL;
    const int n_cols = (2 * N + 15) / 16 * 16;
    const int es = mode == PCAL_DFT_TC_TF32X3 ? 4 : 2;
    const int k_chunks = (2 * N + kChunkBytes / es - 1) / (kChunkBytes / es);
    if (tile < 0 || tile * tile_cols(mode) >= n_cols || chunk < 0 || chunk >= k_chunks) return PCAL_EINVAL;
    double* tw = new (std::nothrow) double[2 * (size_t)N];
    if (!tw) return PCAL_ENOMEM;
    twiddles(N, tw, tw + N);
    *rows = build_weight_tile(N, mode, tile, chunk, tw, tw + N, static_cast<uint8_t*>(hi), static_cast<uint8_t*>(lo));
    delete[] tw;
    return PCAL_OK;
}

extern "C" int pcal_dft_create(int N, int mode, pcal_dft** out) {
    if (!out || N < 1 || N > PCAL_BATCH_MAX_N) return PCAL_EINVAL;
    if (mode != PCAL_DFT_FP32 && mode != PCAL_DFT_TC_TF32X3 && mode != PCAL_DFT_TC_BF16X3) return PCAL_EINVAL;
    pcal_dft* d = new (std::nothrow) pcal_dft();
    if (!d) return PCAL_ENOMEM;
    memset(static_cast<void*>(d), 0, sizeof(*d));
    d->N = N;
    d->mode = mode;
    d->n_cols = (2 * N + 15) / 16 * 16;
    d->col_tiles = mode == PCAL_DFT_FP32 ? 0 : (d->n_cols + tile_cols(mode) - 1) / tile_cols(mode);
    const int es = mode == PCAL_DFT_TC_TF32X3 ? 4 : 2;
    d->k_chunks = (2 * N + kChunkBytes / es - 1) / (kChunkBytes / es);
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
        const int NT = tile_cols(mode), kBTile = NT * kChunkBytes;
        const size_t bytes = (size_t)d->col_tiles * d->k_chunks * 2 * kBTile;
        uint8_t* h = new (std::nothrow) uint8_t[bytes];
        if (!h) e = cudaErrorMemoryAllocation;
        for (int t = 0; h && t < d->col_tiles; ++t)
            for (int kc = 0; kc < d->k_chunks; ++kc) {
                // hi rows, then the lo rows right after them: one copy per chunk
                uint8_t* base = h + ((size_t)t * d->k_chunks + kc) * 2 * kBTile;
                const int rows = build_weight_tile(N, mode, t, kc, tw, tw + N, base, base + kBTile);
                if (rows < NT) memmove(base + (size_t)rows * kChunkBytes, base + kBTile, (size_t)rows * kChunkBytes);
            }
        if (e == cudaSuccess) e = cudaMalloc(&d->d_w, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(d->d_w, h, bytes, cudaMemcpyHostToDevice);
        delete[] h;
    }
    delete[] tw;
    if (e == cudaSuccess && mode != PCAL_DFT_FP32) {
        const int smem = TcCfg<PCAL_DFT_TC_TF32X3>::kSmem;
        static_assert(TcCfg<PCAL_DFT_TC_TF32X3>::kSmem == TcCfg<PCAL_DFT_TC_BF16X3>::kSmem, "one attribute value");
        e = mode == PCAL_DFT_TC_TF32X3
                ? cudaFuncSetAttribute(dft_tc_kernel<PCAL_DFT_TC_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem)
                : cudaFuncSetAttribute(dft_tc_kernel<PCAL_DFT_TC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
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
    const size_t need = (size_t)((C + kTcM - 1) / kTcM) * d->k_chunks * 2 * kATile;
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
    if ((size_t)m_tiles * d->k_chunks * 2 * kATile > d->a_cap) return cudaErrorInvalidValue;  // dft_reserve first
    const int64_t words = m_tiles * d->k_chunks * kImageWords;  // one thread per word (hi and lo)
    const int64_t blocks = (words + 255) / 256;
    const int sgrid = (int)(blocks < 32 * 152 ? blocks : 32 * 152);
    uint4* a_words = reinterpret_cast<uint4*>(d->d_a);
    if (d->mode == PCAL_DFT_TC_TF32X3)
        split_p_kernel<PCAL_DFT_TC_TF32X3><<<sgrid, 256, 0, s>>>(P, C, d->N, d->k_chunks, a_words, words);
    else
        split_p_kernel<PCAL_DFT_TC_BF16X3><<<sgrid, 256, 0, s>>>(P, C, d->N, d->k_chunks, a_words, words);
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
        dft_tc_kernel<PCAL_DFT_TC_BF16X3><<<grid, kTcThreads, TcCfg<PCAL_DFT_TC_BF16X3>::kSmem, s>>>(a);
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
