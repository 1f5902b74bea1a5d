// Bulk fold kernels of libpcal (paper Sec. 2, Eq. 2 with the period L of
// Eq. 4, folded before rotating as in Sec. 4.1's long-accumulator remark).
//
// Layout.  The body of an accumulate call is viewed as a 2-D array of rows:
// each row is `row_samples` samples, a whole number of periods L and of
// 16-byte vectors, so word c of every row always carries the same bins
// (k_a + spw*c + j) mod L, j < spw (spw = samples per 32-bit word).  The grid
// tiles this array by (column group, row group): a CTA owns C_w columns of
// rows_per_cta consecutive rows, and each of its consumer threads owns ONE
// column (word position) and a fixed subset of the rows (replica q of r takes
// rows q, q+r, q+2r, ...).  A thread's bins therefore never change, and it
// keeps its statistics in registers until the end.
//
// Movement.  One producer thread streams the CTA's tile through a ring of
// shared-memory stages with 2-D TMA copies (cp.async.bulk.tensor, tensor map
// over the rows; rows past the end read as zeros, which add nothing), paced
// by full/empty mbarriers.  Every wait is bounded: a wait that gives up sets
// a flag in the plan's device error word and the CTA drains and exits.
//
// Arithmetic per format:
//   2-bit  bit-sliced positional popcounts of the l bits, the h bits and the
//          (h AND l) bits (bitplane.cuh), about 8 integer ops per 16 samples;
//   int8   four IDP4A per word into exact 32-bit sums;
//   f32    Neumaier-compensated FP32 sums.
// At the end each CTA merges its replicas in shared memory and adds its
// integer bins to the plan's accumulators with global atomics (order-free,
// exact); float32 tiles write fixed-order partials that a second kernel sums
// per bin in a fixed order, so float results are deterministic.
#include <stdio.h>
#include <string.h>

#include <cudaTypedefs.h>

#include "bitplane.cuh"
#include "df64.cuh"
#include "internal.cuh"
#include "ptx.cuh"

namespace {

constexpr int kMaxBlock = 640;           // consumer warps + producer warp (<= 96 registers)
constexpr int kSmemBudget = 220 * 1024;  // dynamic shared memory per CTA
constexpr size_t kExclusiveSmem = 200 * 1024;  // the least a fold CTA asks for (see bulk_tiling)

struct BulkArgs {
    int cols_total;   // words per row
    int col_width;    // C_w
    int col_groups;   // G_c
    int replicas;     // r consumer groups
    int wpr;          // warps per group = ceil(col_width / 32)
    int merge_stride; // words between merge rows (col_width rounded up, +2)
    int box_rows;     // rows per stage
    int stages;
    int consumers;    // C_w * r
    uint32_t stage_stride;  // bytes between stages (1024-aligned)
    uint32_t tx_bytes;      // bytes one TMA box delivers
    int total_boxes;  // boxes per column group
    int row_groups;   // CTAs per column group
    int static_boxes; // boxes each CTA takes without the shared counter
    int max_boxes;    // cap per CTA (keeps per-CTA counts below 2^16)
    int chunk;        // boxes per grab from the shared counter
    unsigned long long* sched;  // per column group: (epoch << 32) | boxes handed out
    unsigned int epoch;         // this launch's epoch (never 0)
    int64_t n_rows;
    int64_t k_a;      // phase of the first sample of row 0
    int64_t L;
    unsigned long long* acc2;
    long long* acc8;
    float2* partf;    // f32: [row group][cols_total] partial sums
    unsigned int* err;
    const PrefetchHint* hint;   // the plan's hint ring (launch epoch + 1 is the next launch)
};

using namespace pcal_ptx;

// Pull the first rows of the next launch's row groups rg, rg + row_groups,
// ... into L2, from the ring record of epoch + 1 loaded at the start (w0-w2);
// nothing unless all three words carry that launch's tag.  The rows of a
// group are one contiguous range; the CTAs of this launch's column groups
// take equal slices of it (cg of col_groups), so every CTA issues a few
// prefetches.  Rows stay inside that launch's input.
__device__ __noinline__ void prefetch_next_launch(const BulkArgs& a, int64_t rg, int cg, unsigned long long w0,
                                                  unsigned long long w1, unsigned long long w2) {
    const unsigned long long tag = hint_tag((unsigned long long)a.epoch + 1ull);
    if ((w0 >> 48) != tag || (w1 >> 48) != tag || (w2 >> 48) != tag) return;
    constexpr unsigned long long kLow48 = (1ull << 48) - 1, kPiece = 32768;
    const unsigned long long n_rows = w0 & kLow48, base = (w1 & kLow48) << 4;
    const unsigned long long groups = (w2 >> 32) & 0xffffu, group_rows = (w2 >> 16) & 0xffffu,
                             first_rows = w2 & 0xffffu;
    const unsigned long long row_bytes = 4ull * (unsigned long long)a.cols_total;
    for (unsigned long long r2 = (unsigned long long)rg; r2 < groups; r2 += (unsigned long long)a.row_groups) {
        const unsigned long long row0 = r2 * group_rows;
        if (row0 >= n_rows) break;
        const unsigned long long rows = first_rows < n_rows - row0 ? first_rows : n_rows - row0;
        const unsigned long long addr = base + row0 * row_bytes, bytes = rows * row_bytes;
        const unsigned long long gcs = (unsigned long long)a.col_groups;
        const unsigned long long o0 = bytes * (unsigned long long)cg / gcs / 16 * 16;
        const unsigned long long o1 = (unsigned long long)cg + 1 == gcs ? bytes : bytes * (cg + 1ull) / gcs / 16 * 16;
        for (unsigned long long off = o0; off < o1; off += kPiece)
            prefetch_l2(addr + off, (uint32_t)(o1 - off < kPiece ? o1 - off : kPiece));
    }
}

// ---- per-format consumer state --------------------------------------------------

template <int U>
struct Acc2 {
    // w stream: planes of weight 1..16 + U upper planes (weight 32 on);
    // d stream: planes of weight 1..8 + U upper planes (weight 16 on).
    uint32_t w1 = 0, w2 = 0, w4 = 0, w8 = 0, w16 = 0, wu[U];
    uint32_t d1 = 0, d2 = 0, d4 = 0, d8 = 0, du[U];
    __device__ Acc2() {
#pragma unroll
        for (int u = 0; u < U; ++u) wu[u] = du[u] = 0;
    }
    // 32 words of this thread's column, from 32 of its rows.
    __device__ __forceinline__ void add32(const uint32_t (&x)[32]) {
        pcal_bits::add32<U>(x, w1, w2, w4, w8, w16, wu, d1, d2, d4, d8, du);
    }
};

struct Acc8 {
    int s[4] = {0, 0, 0, 0};
    __device__ __forceinline__ void add(uint32_t w) {
        s[0] = __dp4a((int)w, 0x00000001, s[0]);
        s[1] = __dp4a((int)w, 0x00000100, s[1]);
        s[2] = __dp4a((int)w, 0x00010000, s[2]);
        s[3] = __dp4a((int)w, 0x01000000, s[3]);
    }
};

struct AccF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(uint32_t w) {
        const float x = __uint_as_float(w);
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
};

// Hand out `take` boxes of a column group: the counter word is (epoch << 32)
// | boxes handed out.  The first grab of a launch finds an older epoch and
// swaps in (epoch, 0); no launch touches the word after its CTAs have started
// the next launch (they trigger it only once their grabs are done), so no
// reset is needed.  Returns the first box, or -1 on an inconsistent word.
__device__ int grab_boxes(unsigned long long* ctr, unsigned int epoch, int take, unsigned int* err) {
    const unsigned long long mine = (unsigned long long)epoch << 32;
    unsigned long long cur = atomicAdd(ctr, 0ull);
    for (int i = 0; (unsigned int)(cur >> 32) != epoch; ++i) {
        if (i > 1024) {
            atomicOr(err, PCAL_DERR_SCHED);
            return -1;
        }
        const unsigned long long prev = atomicCAS(ctr, cur, mine);
        cur = prev == cur ? mine : prev;
    }
    const unsigned long long r = atomicAdd(ctr, (unsigned long long)take);
    if ((unsigned int)(r >> 32) != epoch) {
        atomicOr(err, PCAL_DERR_SCHED);
        return -1;
    }
    return (int)(r & 0xffffffffull);
}

// ---- the kernel ------------------------------------------------------------------
// FMT: PCAL_2BIT, PCAL_I8 or PCAL_F32.  U: upper bit planes (2-bit only).
//
// Threads: `replicas` groups of `wpr` consumer warps, then one producer warp.
// Lane c < col_width of a group owns column c0 + c; group q consumes the
// boxes q, q + r, q + 2r, ... whole.  Box j lives in stage j % stages, and
// stages is a multiple of r, so every stage belongs to one group, which
// waits for its uses in order.  Every thread of the group arrives on the
// stage's empty barrier once it holds the box's words in registers (2-bit)
// or has folded them (int8, float32).
template <int FMT, int U>
__global__ void __launch_bounds__(kMaxBlock, 1) bulk_fold_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                 const BulkArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x;
    const int group_threads = a.wpr * 32;
    const int n_cons_warps = a.wpr * a.replicas;
    const int producer_warp = n_cons_warps;
    const int cg = blockIdx.x % a.col_groups;
    const int64_t rg = blockIdx.x / a.col_groups;
    const int c0 = cg * a.col_width;

    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)a.stages * a.stage_stride);
    uint64_t* empty = full + a.stages;
    __shared__ int s_failed;
    __shared__ int s_end;          // local box index where this CTA's work ends
    __shared__ int s_last_fill[8]; // per stage: local index of its last TMA fill, or -1
    __shared__ int s_fill_open[8]; // per stage: that fill is the stage's latest phase

    if (tid == 0) {
        s_failed = 0;
        s_end = 0x7fffffff;
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], group_threads);
            s_last_fill[s] = -1;
            s_fill_open[s] = 0;
        }
        fence_barrier_init();
    }
    __syncthreads();

    const int q = tid / group_threads;   // replica group
    const int col = tid % group_threads; // column within the tile
    const bool active = tid < n_cons_warps * 32 && col < a.col_width;
    Acc2<(FMT == PCAL_2BIT ? U : 1)> acc2;
    Acc8 acc8;
    AccF accf;

    if (tid / 32 == producer_warp) {
        // ---------------- producer ----------------
        // Boxes: a static share first (no atomics on the start-up path),
        // then chunks from the column group's counter until the work or the
        // per-CTA cap runs out.  Local box j goes to stage j % stages.
        if (tid % 32 == 0) {
            // the samples are read once: their L2 lines go first, so the
            // stream does not evict the bins and tables the finalize reuses
            const uint64_t policy = l2_policy_evict_first();
            // the next launch's read start (used at the end; loaded now so
            // that the latency of host memory hides behind the first copies)
            unsigned long long hint0 = 0, hint1 = 0, hint2 = 0;
            if (a.hint) {
                const PrefetchHint* h = a.hint + (((unsigned long long)a.epoch + 1ull) % kHintRing);
                hint0 = ld_relaxed_sys(&h->rows);
                hint1 = ld_relaxed_sys(&h->base);
                hint2 = ld_relaxed_sys(&h->groups);
            }
            int j = 0;
            bool ok = true;
            auto stage_free = [&](int jj) -> bool {
                const int s = jj % a.stages;
                const uint32_t use = jj / a.stages;
                if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
                    atomicOr(a.err, PCAL_DERR_EMPTY_WAIT);
                    s_failed = 1;
                    return false;
                }
                return true;
            };
            auto issue = [&](int box) -> bool {
                if (!stage_free(j)) return false;
                const int s = j % a.stages;
                mbar_arrive_expect_tx(&full[s], a.tx_bytes);
                tma_load_2d_hint(smem + (size_t)s * a.stage_stride, &tmap, c0, box * a.box_rows, &full[s], policy);
                s_last_fill[s] = j;
                s_fill_open[s] = 1;
                ++j;
                return true;
            };
            for (int b = 0; b < a.static_boxes && ok; ++b) {
                const int box = (int)rg * a.static_boxes + b;
                if (box >= a.total_boxes) break;
                ok = issue(box);
            }
            const int base = a.row_groups * a.static_boxes;
            while (ok && j < a.max_boxes) {
                const int take = a.chunk < a.max_boxes - j ? a.chunk : a.max_boxes - j;
                const int v = grab_boxes(&a.sched[cg], a.epoch, take, a.err);
                if (v < 0) {
                    s_failed = 1;
                    ok = false;
                    break;
                }
                if (base + v >= a.total_boxes) break;
                for (int c = 0; c < take && ok && base + v + c < a.total_boxes; ++c) ok = issue(base + v + c);
            }
            // end of work: every group gets a data-less phase on the next
            // stage it owns, after which it reads s_end and stops
            if (ok) {
                s_end = j;
                for (int g = 0; g < a.replicas && ok; ++g) {
                    int jq = j;
                    while (jq % a.replicas != g) ++jq;
                    if (!stage_free(jq)) {
                        ok = false;
                        break;
                    }
                    s_fill_open[jq % a.stages] = 0;
                    mbar_arrive(&full[jq % a.stages]);
                }
            }
            // This CTA grabs no more boxes: once every CTA is here the next
            // launch may start (its CTAs take the SMs as this launch's CTAs
            // leave, and the shared counters are free for its new epoch).
            // The consumers still have the stages in flight to fold.
            allow_dependents();
            if (a.hint) prefetch_next_launch(a, rg, cg, hint0, hint1, hint2);
        }
    } else {
        // ---------------- consumers ----------------
        for (int j = q;; j += a.replicas) {
            const int s = j % a.stages;
            const uint32_t use = j / a.stages;
            if (!mbar_wait(&full[s], use & 1)) {
                atomicOr(a.err, PCAL_DERR_FULL_WAIT);
                s_failed = 1;
                break;
            }
            if (j >= *reinterpret_cast<volatile int*>(&s_end)) break;
            const uint32_t* p = reinterpret_cast<const uint32_t*>(smem + (size_t)s * a.stage_stride) + col;
            if (FMT == PCAL_2BIT) {
                for (int b = 0; b < a.box_rows; b += 32) {
                    uint32_t x[32];
                    if (active) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) x[i] = p[i * a.col_width];
                    }
                    p += 32 * a.col_width;
                    if (b + 32 >= a.box_rows) mbar_arrive(&empty[s]);  // words are in registers
                    if (active) acc2.add32(x);
                }
            } else {
                if (active) {
                    if (FMT == PCAL_I8) {
#pragma unroll 8
                        for (int i = 0; i < a.box_rows; ++i) acc8.add(p[i * a.col_width]);
                    } else {
#pragma unroll 8
                        for (int i = 0; i < a.box_rows; ++i) accf.add(p[i * a.col_width]);
                    }
                }
                mbar_arrive(&empty[s]);
            }
        }
    }
    __syncthreads();
    // Every grab of this CTA is done (the producer signalled it already): the
    // next launch in the stream may start (a finalize waits for this kernel;
    // a fold uses a new counter epoch and adds into the same bins with
    // atomics, or into the other bin set).
    allow_dependents();
    if (s_failed) {
        // Drain: TMA fills whose phase no consumer waited for must land
        // before the CTA exits (its shared memory is then reused).
        if (tid == 0)
            for (int s = 0; s < a.stages; ++s)
                if (s_fill_open[s] && s_last_fill[s] >= 0 &&
                    !mbar_wait(&full[s], (uint32_t)(s_last_fill[s] / a.stages) & 1))
                    atomicOr(a.err, PCAL_DERR_DRAIN_WAIT);
        grid_dependency_wait();
        return;
    }

    // ---------------- merge replicas, then flush ----------------
    // The stage buffers are free now (every fill landed and was consumed);
    // they hold the merge scratch.  Layouts keep consecutive lanes on
    // consecutive words (no bank conflicts).
    if (FMT == PCAL_2BIT) {
        uint32_t W[16], D[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) W[i] = D[i] = 0;
        W[0] = acc2.w1;
        W[1] = acc2.w2;
        W[2] = acc2.w4;
        W[3] = acc2.w8;
        W[4] = acc2.w16;
        D[0] = acc2.d1;
        D[1] = acc2.d2;
        D[2] = acc2.d4;
        D[3] = acc2.d8;
#pragma unroll
        for (int u = 0; u < (FMT == PCAL_2BIT ? U : 1); ++u) {
            if (5 + u < 16) W[5 + u] = acc2.wu[u];
            if (4 + u < 16) D[4 + u] = acc2.du[u];
        }
        // Replicas add up in the bit-plane domain (ripple-carry adds of
        // 16-plane numbers; per-CTA counts stay below 2^16): group 0 gathers
        // the l/h planes W, group 1 the (h AND l) planes D, and each of the two
        // transposes its planes into counts, so the work splits in half.
        // scratch[(i*r + q)*C_w + col], i < 32 (16 W planes, 16 D planes)
        uint32_t* scratch = reinterpret_cast<uint32_t*>(smem);
        const int rc = a.replicas * a.col_width;
        const int qd = a.replicas > 1 ? 1 : 0;  // the group that gathers D
        if (active) {
            uint32_t* dst = scratch + q * a.col_width + col;
            if (q != 0)
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[i * rc] = W[i];
            if (q != qd)
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[(16 + i) * rc] = D[i];
        }
        __syncthreads();
        uint32_t* m = scratch + 32 * rc;  // counts of column col: m[i*S + col], i < 32
        if (active && (q == 0 || q == qd)) {
            for (int o = 0; o < a.replicas; ++o) {
                if (o == q) continue;
                const uint32_t* src = scratch + o * a.col_width + col;
                if (q == 0) {
                    uint32_t c = 0;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const uint32_t b = src[i * rc];
                        const uint32_t sum = pcal_bits::lop3<pcal_bits::kXor3>(W[i], b, c);
                        c = pcal_bits::lop3<pcal_bits::kMaj3>(W[i], b, c);
                        W[i] = sum;
                    }
                }
                if (q == qd) {
                    uint32_t c = 0;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const uint32_t b = src[(16 + i) * rc];
                        const uint32_t sum = pcal_bits::lop3<pcal_bits::kXor3>(D[i], b, c);
                        c = pcal_bits::lop3<pcal_bits::kMaj3>(D[i], b, c);
                        D[i] = sum;
                    }
                }
            }
            if (q == 0) {
                pcal_bits::transpose16x2(W);
#pragma unroll
                for (int i = 0; i < 16; ++i) m[i * a.merge_stride + col] = W[i];
            }
            if (q == qd) {
                pcal_bits::transpose16x2(D);
#pragma unroll
                for (int i = 0; i < 16; ++i) m[(16 + i) * a.merge_stride + col] = D[i];
            }
        }
        __syncthreads();
        // The bins this fold adds into were cleared by the finalize two
        // kernels back; waiting for the preceding kernel here (it waited for
        // its own predecessor) orders these atomics after that clearing.
        grid_dependency_wait();
        // one atomic per (column, sample): consecutive threads, consecutive
        // bins; each row group starts at its own offset, so that the CTAs
        // flushing at the same time spread over the bins.  bin = (k_a + 16 gc
        // + j) mod L = (base + t) mod L with base + t < L + 2^12 (L <= 2^20).
        const int S = a.merge_stride;
        const int tasks = a.col_width * 16;
        const uint32_t Lu = (uint32_t)a.L;
        const uint32_t base = (uint32_t)((a.k_a + 16 * (int64_t)c0) % a.L);
        const int rot = (int)(rg * tasks / a.row_groups);  // rg < row_groups
        for (int t0 = tid; t0 < tasks; t0 += blockDim.x) {
            const int t = t0 + rot < tasks ? t0 + rot : t0 + rot - tasks;
            const int cl = t >> 4, j = t & 15;
            const int gc = c0 + cl;
            if (gc >= a.cols_total) continue;
            const int pl = 2 * j, ph = 2 * j + 1;  // bit positions of l and h
            const uint32_t sl = (m[(pl & 15) * S + cl] >> (16 * (pl >> 4))) & 0xFFFFu;
            const uint32_t sh = (m[(ph & 15) * S + cl] >> (16 * (ph >> 4))) & 0xFFFFu;
            const uint32_t shl = ((m[(16 + (pl & 15)) * S + cl] >> (16 * (pl >> 4))) & 0xFFFFu) +
                                 ((m[(16 + (ph & 15)) * S + cl] >> (16 * (ph >> 4))) & 0xFFFFu);
            if ((sl | sh) == 0) continue;
            uint32_t bin = base + (uint32_t)t;
            if (bin >= Lu) bin -= Lu;
            if (bin >= Lu) bin %= Lu;
            atomicAdd(&a.acc2[bin], (unsigned long long)sl | ((unsigned long long)sh << 21) |
                                         ((unsigned long long)shl << 42));
        }
    } else if (FMT == PCAL_I8) {
        // m[j*S + col], j < 4
        int* m = reinterpret_cast<int*>(smem);
        const int S = a.merge_stride;
        for (int i = tid; i < 4 * S; i += blockDim.x) m[i] = 0;
        __syncthreads();
        if (active) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (acc8.s[j]) atomicAdd(&m[j * S + col], acc8.s[j]);
        }
        __syncthreads();
        grid_dependency_wait();  // as for the 2-bit flush
        const int tasks = a.col_width * 4;
        const uint32_t Lu = (uint32_t)a.L;
        const uint32_t base = (uint32_t)((a.k_a + 4 * (int64_t)c0) % a.L);
        const int rot = (int)(rg * tasks / a.row_groups);  // rg < row_groups
        for (int t0 = tid; t0 < tasks; t0 += blockDim.x) {
            const int t = t0 + rot < tasks ? t0 + rot : t0 + rot - tasks;
            const int cl = t >> 2, j = t & 3;
            const int gc = c0 + cl;
            const int v = m[j * S + cl];
            if (gc >= a.cols_total || v == 0) continue;
            uint32_t bin = base + (uint32_t)t;
            if (bin >= Lu) bin -= Lu;
            if (bin >= Lu) bin %= Lu;
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.acc8[bin]), (unsigned long long)(long long)v);
        }
    } else {
        // f32: replicas in a fixed order, then one partial per column per
        // row group; a second kernel sums the partials per bin.
        float2* m = reinterpret_cast<float2*>(smem);
        if (active) m[q * a.col_width + col] = make_float2(accf.s, accf.c);
        __syncthreads();
        // the partials of the previous f32 launch are summed by its reduce
        // kernel, which may still run: wait for the preceding kernel first
        grid_dependency_wait();
        if (tid < a.col_width && c0 + tid < a.cols_total) {
            float s = 0.f, c = 0.f;
            for (int r = 0; r < a.replicas; ++r) {
                const float2 v = m[r * a.col_width + tid];
                const float t = s + v.x;
                c += (fabsf(s) >= fabsf(v.x) ? (s - t) + v.x : (v.x - t) + s) + v.y;
                s = t;
            }
            a.partf[rg * a.cols_total + c0 + tid] = make_float2(s, c);
        }
    }
    // This kernel only completes after the preceding one has, so the
    // completion order of the stream's kernels stays the launch order (a
    // second wait returns at once).
    grid_dependency_wait();
}

// f32: bin k += the sum over the pending slots, their row groups and the
// columns that map to k, in a fixed order and in double-float.  One warp per
// bin: lane j sums terms j, j + 32, ... (slot, then row group major), then a
// fixed shuffle tree adds the lanes, so the partials are loaded 32 at a time
// (a thread per bin waited out 19 dependent L2 loads per slot on a 64 MB
// input) and the result does not depend on timing.  Launched as a
// programmatic dependent of the preceding kernel: it lets the next kernel
// start launching, then waits for the partials.  The next kernel can launch
// only once every block of this one has started, so the grid is at most one
// block per SM and its warps stride over the bins.
constexpr int kReduceWarps = 16;  // warps per block

struct PendingArgs {
    const float2* base[kPartSlots];
    int64_t row_groups[kPartSlots];
    int64_t k_a[kPartSlots];
    int n;
};

// The slot arguments are indexed at run time: as a grid constant they are
// read in place (a by-value parameter was copied to every thread's stack,
// 104 B x 512 threads per block: megabytes of dirty L2 lines per flush that
// the next fold had to write back).
__global__ void __launch_bounds__(32 * kReduceWarps) reduce_f32_kernel(const __grid_constant__ PendingArgs pa, int cols_total,
                                                                      int64_t L, float2* __restrict__ acc) {
    allow_dependents();
    grid_dependency_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * kReduceWarps;
    for (int64_t k = blockIdx.x * (int64_t)kReduceWarps + threadIdx.x / 32; k < L; k += warps) {
        pcal_df::df s{0.f, 0.f};
        for (int e = 0; e < pa.n; ++e) {
            const int64_t c_first = ((k - pa.k_a[e]) % L + L) % L;
            if (c_first >= cols_total) continue;  // whole warps skip together
            const int64_t per_rg = (cols_total - 1 - c_first) / L + 1;  // columns of this bin in a row
            const int64_t terms = pa.row_groups[e] * per_rg;
            for (int64_t t = lane; t < terms; t += 32) {
                const int64_t rg = t / per_rg, c = c_first + (t % per_rg) * L;
                const float2 v = pa.base[e][rg * cols_total + c];
                s = pcal_df::add(s, pcal_df::two_sum(v.x, v.y));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const pcal_df::df o{__shfl_down_sync(0xffffffffu, s.hi, off),
                                __shfl_down_sync(0xffffffffu, s.lo, off)};
            s = pcal_df::add(s, o);
        }
        if (lane == 0) {
            const float2 a = acc[k];
            s = pcal_df::add(pcal_df::df{a.x, a.y}, s);
            acc[k] = make_float2(s.hi, s.lo);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int bits_for(int64_t v) {
    int b = 0;
    while (((int64_t)1 << b) <= v) ++b;
    return b;
}

// Launched as a programmatic dependent of the preceding kernel: its CTAs may
// start while that kernel finishes.  Nothing it touches depends on that
// kernel (new counter epoch; atomics into the current bin set, which a
// preceding finalize does not touch); it waits for it only at its very end.
template <int FMT, int U>
cudaError_t launch_one(const CUtensorMap& map, const BulkArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
    auto k = bulk_fold_kernel<FMT, U>;
    static size_t smem_set = 0;  // per instantiation; the attribute only grows
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, map, a);
}

}  // namespace

int bulk_tiling(const pcal_plan* p, int64_t n_rows, BulkTiling* t) {
    const int spw = p->g.samples_per_byte_x4;
    const int cols = (int)(p->g.row_samples / spw);
    BulkTiling z{};
    z.cols_total = cols;
    // column groups of at most 256 words (the TMA box limit), 32-byte wide
    const int sms_fold = p->num_sms >= 64 ? p->num_sms - kFinalizeReserveSms : p->num_sms;
    int gc = (cols + 255) / 256;
    int cw = (cols + gc - 1) / gc;
    cw = (cw + 7) / 8 * 8;
    if (cw > 256) cw = 256;
    gc = (cols + cw - 1) / cw;
    // Wide rows (long periods): few row groups per column group leave SMs
    // idle (e.g. 50 groups x 2 rows on 136 SMs); narrow the groups until the
    // CTAs fill at least 90 % of a whole number of waves.
    for (int g = gc; cw > 32; ++g) {
        const int w = ((cols + g - 1) / g + 7) / 8 * 8;
        const int gg = (cols + w - 1) / w;
        const int rows_per = sms_fold / gg > 0 ? sms_fold / gg : 1;
        const int ctas = gg * rows_per;
        const int waves = (ctas + sms_fold - 1) / sms_fold;
        if (10 * ctas >= 9 * waves * sms_fold) {
            cw = w;
            gc = gg;
            break;
        }
        if (w <= 32) break;
    }
    // An even cut where one exists: equal column groups stream equal bytes
    // (work is balanced within a column group, not across them; C1 float32:
    // 7 groups of 232 words left the 208-word group's CTAs idle at the end,
    // 8 of 200 fill 136 CTAs), if it fills the SMs at least as well.
    {
        auto fill = [&](int g) { return g * (sms_fold / g > 0 ? sms_fold / g : 1); };
        for (int g = gc; g <= 2 * gc && g <= cols; ++g) {
            if (cols % g != 0 || (cols / g) % 8 != 0 || cols / g > 256) continue;
            if (g == gc && cols / g == cw) break;  // already even
            if (fill(g) >= fill(gc)) {
                gc = g;
                cw = cols / g;
            }
            break;
        }
    }
    z.col_width = cw;
    z.col_groups = gc;
    const int wpr = (cw + 31) / 32;
    int r_max = (kMaxBlock / 32 - 1) / wpr;
    if (r_max > 8) r_max = 8;
    if (r_max < 1) r_max = 1;
    // 2-bit and float32: a stage of about 48-64 KB (2-bit: whole 32-row
    // blocks).  Each TMA box copy costs the producer a fixed ~0.3 us to issue
    // under load, whatever its size, so fewer, larger boxes keep up with the
    // consumers and fill the pipeline sooner after a launch (float32 C1:
    // 22 KB boxes held a CTA to ~48 GB/s, 51 KB boxes took the fold from
    // 12.95 to 12.28 us).  int8: about 24-32 KB, which keeps 2 replica groups
    // and 8 stages on wide rows (its 1 GiB folds run at 0.98 of the copy
    // bandwidth).
    const int unit = p->g.format == PCAL_2BIT ? 32 : 8;
    int units = (p->g.format != PCAL_I8 ? 56 * 1024 : 28 * 1024) / (unit * cw * 4);
    if (units < 1) units = 1;
    int box = unit * units;
    while (box > 256) box -= unit;
    z.box_rows = box;
    const size_t stage = (size_t)box * cw * 4;
    const size_t stage_al = (stage + 1023) / 1024 * 1024;
    // Box j lives in stage j % stages and is consumed by group j % r.  With
    // stages a multiple of r every stage belongs to ONE group, which waits
    // for its uses in order; otherwise a fast group could wait on a stage
    // two phases ahead, where the mbarrier parity test would match an older
    // phase (wrong tile, and arrivals beyond the barrier's count).
    int r = 0, stages = 0;
    const int ms = (cw + 31) / 32 * 32 + 2;  // merge stride
    for (int rr = r_max; rr >= 1 && r == 0; --rr) {
        int st = (int)((kSmemBudget - 1024) / stage_al);
        if (st > 8) st = 8;
        st = st / rr * rr;
        if (st < 3 || st < rr) continue;
        // after the main loop the stage buffers hold the merge scratch
        const size_t need = p->g.format == PCAL_2BIT ? (size_t)128 * rr * cw + (size_t)128 * ms
                            : (p->g.format == PCAL_I8 ? (size_t)16 * ms : (size_t)8 * rr * cw);
        if (need > (size_t)st * stage_al) continue;
        r = rr;
        stages = st;
    }
    if (r == 0) return -1;
    z.replicas = r;
    z.stages = stages;
    z.merge_stride = ms;
    // Work split: boxes of one column group are shared by row_groups CTAs
    // (one wave over the SMs the finalize does not need): a static share
    // each, the rest handed out in chunks from a counter; each CTA takes at
    // most max_boxes (twice the average), which keeps its 16-bit
    // per-position counts below 2^16.
    const int64_t total = (n_rows + box - 1) / box;
    if (total > 0x3fffffff) return -1;
    const int64_t cap = 65535 / box;
    int64_t gr = sms_fold / gc;
    if (gr < 1) gr = 1;
    if (gr > total) gr = total;
    while ((total + gr - 1) / gr * 2 > cap) ++gr;  // very long inputs: more CTAs
    const int64_t avg = (total + gr - 1) / gr;
    int64_t maxb = 2 * avg;
    if (maxb > cap) maxb = cap;
    const int64_t stat = avg < 16 ? avg * 7 / 8 : avg * 3 / 4;  // (short folds: see the grab size below)
    z.row_groups = gr;
    z.total_boxes = (int)total;
    z.static_boxes = (int)stat;
    z.max_boxes = (int)maxb;
    // boxes per grab: 4 (2 -> 4: C2 -0.2 us per step, 1 GiB int8 launches
    // 181 -> 164 us), but 2 when a CTA has fewer than 16 boxes on average,
    // with 7/8 of them static, so the last grabs end closer together (C1
    // float32, 9 boxes per CTA: fold 11.96 -> 11.6 us; one box at a time or
    // half the boxes static: slower)
    z.chunk = avg < 16 ? 2 : 4;
    z.rows_per_cta = maxb * box;  // the most rows one CTA can fold
    z.upper_planes = 0;
    if (p->g.format == PCAL_2BIT) {
        const int64_t rows_per_thread = (maxb + r - 1) / r * box;
        z.upper_planes = bits_for(rows_per_thread / 32);
    }
    z.threads = (wpr * r + 1) * 32;
    z.smem_bytes = (size_t)stages * stage_al + 16 * (size_t)stages;
    // A fold CTA takes at least kExclusiveSmem, so that no CTA of the finalize
    // that overlaps the fold fits beside it (sharing an SM with a fold CTA
    // slows the finalize 2-3x; float32 tilings of ~180 KB let it in: C1 step
    // 20.95 -> 19.96 us with the floor).
    if (z.smem_bytes < kExclusiveSmem) z.smem_bytes = kExclusiveSmem;
    *t = z;
    return 0;
}

namespace {

// A launch that failed to enqueue takes its published read start back: the
// launch before it must not pull rows of a buffer nothing will read.
void unpublish_hint(pcal_plan* p, unsigned int epoch) {
    if (!p->h_hint) return;
    PrefetchHint* h = p->h_hint + (epoch % kHintRing);
    __atomic_store_n(&h->rows, 0ull, __ATOMIC_RELAXED);
    __atomic_store_n(&h->base, 0ull, __ATOMIC_RELAXED);
    __atomic_store_n(&h->groups, 0ull, __ATOMIC_RELAXED);
}

}  // namespace

cudaError_t flush_partials(pcal_plan* p, cudaStream_t s) {
    if (p->g.format != PCAL_F32 || p->n_pending == 0) return cudaSuccess;
    PendingArgs pa{};
    for (int e = 0; e < p->n_pending; ++e) {
        pa.base[e] = p->pending[e].base;
        pa.row_groups[e] = p->pending[e].row_groups;
        pa.k_a[e] = p->pending[e].k_a;
    }
    pa.n = p->n_pending;
    const int spw = p->g.samples_per_byte_x4;
    const int cols_total = (int)(p->g.row_samples / spw);
    const int64_t blocks = (p->g.L + kReduceWarps - 1) / kReduceWarps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(blocks < p->num_sms ? blocks : p->num_sms));
    cfg.blockDim = dim3(32 * kReduceWarps);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, reduce_f32_kernel, pa, cols_total, (int64_t)p->g.L, cur_accf(p));
    if (e == cudaSuccess) {
        p->n_pending = 0;
        p->stats.kernel_launches += 1;
    }
    return e;
}

cudaError_t launch_bulk(pcal_plan* p, const void* d_rows, int64_t n_rows, int64_t k_a, cudaStream_t s, int* launched) {
    *launched = 0;
    const BulkMapEntry* hit = nullptr;
    for (int i = 0; i < kBulkMapCache; ++i)
        if (p->map_cache[i].ptr == d_rows && p->map_cache[i].rows == n_rows) hit = &p->map_cache[i];
    if (!hit) {
        BulkMapEntry ent{};
        if (bulk_tiling(p, n_rows, &ent.tiling) != 0) return cudaErrorInvalidConfiguration;
        const BulkTiling& t = ent.tiling;
        PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
        if (!enc) return cudaErrorNotSupported;
        const int spw = p->g.samples_per_byte_x4;
        cuuint64_t dims[2] = {(cuuint64_t)t.cols_total, (cuuint64_t)n_rows};
        cuuint64_t strides[1] = {(cuuint64_t)(p->g.row_samples / spw * 4)};
        cuuint32_t box[2] = {(cuuint32_t)t.col_width, (cuuint32_t)t.box_rows};
        cuuint32_t estr[2] = {1, 1};
        // 128-byte L2 promotion (256 B: C2 fold 20.6 us, C1 12.3 us; 128 B or
        // none: 20.5 and 12.0 us; 1 GiB int8 the same either way)
        CUresult r = enc(&ent.map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(d_rows), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        ent.ptr = d_rows;
        ent.rows = n_rows;
        p->map_cache[p->map_next] = ent;
        hit = &p->map_cache[p->map_next];
        p->map_next = (p->map_next + 1) % kBulkMapCache;
    }
    const BulkTiling& t = hit->tiling;
    const CUtensorMap& map = hit->map;
    BulkArgs a{};
    a.cols_total = t.cols_total;
    a.col_width = t.col_width;
    a.col_groups = t.col_groups;
    a.replicas = t.replicas;
    a.wpr = (t.col_width + 31) / 32;
    a.merge_stride = t.merge_stride;
    a.box_rows = t.box_rows;
    a.stages = t.stages;
    a.consumers = a.wpr * 32 * t.replicas;
    a.tx_bytes = (uint32_t)((size_t)t.box_rows * t.col_width * 4);
    a.stage_stride = (a.tx_bytes + 1023u) / 1024u * 1024u;
    a.total_boxes = t.total_boxes;
    a.row_groups = (int)t.row_groups;
    a.static_boxes = t.static_boxes;
    a.max_boxes = t.max_boxes;
    a.chunk = t.chunk;
    a.sched = p->d_sched;
    a.epoch = ++p->bulk_epoch;
    if (a.epoch == 0) a.epoch = ++p->bulk_epoch;  // 0 is the zeroed counters' epoch
    a.n_rows = n_rows;
    a.k_a = k_a;
    a.L = p->g.L;
    a.acc2 = cur_acc2(p);
    a.acc8 = cur_acc8(p);
    a.err = p->d_err;
    a.hint = p->d_hint;
    if (p->h_hint) {
        // publish where this launch starts reading (ring slot of its epoch);
        // a launch whose fields do not fit the packed words publishes nothing
        const unsigned long long base = (unsigned long long)reinterpret_cast<uintptr_t>(d_rows);
        // the successor's first two boxes per CTA (on C2 two gave -0.8 us per step against
        // none; four gave +0.2 us: the prefetch then competes with this launch's own tail)
        const unsigned long long first_rows = (unsigned long long)(t.static_boxes < 2 ? t.static_boxes : 2) * t.box_rows;
        const unsigned long long group_rows = (unsigned long long)t.static_boxes * t.box_rows;
        if ((unsigned long long)n_rows < (1ull << 48) && base < (1ull << 52) && base % 16 == 0 &&
            (unsigned long long)t.row_groups < (1ull << 16) && group_rows < (1ull << 16) && first_rows < (1ull << 16)) {
            const unsigned long long tag = hint_tag(a.epoch) << 48;
            PrefetchHint* h = p->h_hint + (a.epoch % kHintRing);
            __atomic_store_n(&h->rows, tag | (unsigned long long)n_rows, __ATOMIC_RELAXED);
            __atomic_store_n(&h->base, tag | (base >> 4), __ATOMIC_RELAXED);
            __atomic_store_n(&h->groups,
                             tag | ((unsigned long long)t.row_groups << 32) | (group_rows << 16) | first_rows,
                             __ATOMIC_RELAXED);
        }
    }
    const int grid = (int)(t.col_groups * t.row_groups);
    cudaError_t e;
    if (p->g.format == PCAL_F32) {
        // the partials go to the next free slot; they are added into the bins
        // by the finalize (or by a reduce launch when the slots run out)
        const size_t need = (size_t)t.row_groups * t.cols_total;
        e = cudaSuccess;
        if (p->n_pending == kPartSlots || (need > p->partf_cap && p->n_pending > 0)) e = flush_partials(p, s);
        if (e == cudaSuccess && need > p->partf_cap) {
            cudaFree(p->d_partf);  // (waits for the device: no kernel reads the old slots afterwards)
            p->d_partf = nullptr;
            p->partf_cap = 0;
            e = cudaMalloc(&p->d_partf, kPartSlots * need * sizeof(float2));
            if (e == cudaSuccess) p->partf_cap = need;
            p->part_next = 0;
        }
        if (e != cudaSuccess) {
            unpublish_hint(p, a.epoch);
            return e;
        }
        const int slot = p->part_next;
        a.partf = p->d_partf + (size_t)slot * p->partf_cap;
        e = launch_one<PCAL_F32, 1>(map, a, grid, t.threads, t.smem_bytes, s);
        if (e != cudaSuccess) {
            unpublish_hint(p, a.epoch);
            return e;
        }
        p->part_next = (slot + 1) % kPartSlots;
        p->pending[p->n_pending++] = PartSlot{a.partf, (int64_t)t.row_groups, k_a};
        *launched = 1;
        p->stats.kernel_launches += 1;
        return cudaSuccess;
    }
    if (p->g.format == PCAL_I8) {
        e = launch_one<PCAL_I8, 1>(map, a, grid, t.threads, t.smem_bytes, s);
    } else {
        const int u = t.upper_planes;
        if (u <= 3)
            e = launch_one<PCAL_2BIT, 3>(map, a, grid, t.threads, t.smem_bytes, s);
        else if (u <= 5)
            e = launch_one<PCAL_2BIT, 5>(map, a, grid, t.threads, t.smem_bytes, s);
        else if (u <= 7)
            e = launch_one<PCAL_2BIT, 7>(map, a, grid, t.threads, t.smem_bytes, s);
        else if (u <= 9)
            e = launch_one<PCAL_2BIT, 9>(map, a, grid, t.threads, t.smem_bytes, s);
        else
            e = launch_one<PCAL_2BIT, 11>(map, a, grid, t.threads, t.smem_bytes, s);
    }
    if (e == cudaSuccess) {
        *launched = 1;
        p->stats.kernel_launches += 1;
    } else {
        unpublish_hint(p, a.epoch);
    }
    return e;
}

extern "C" int pcal_bulk_tiling(double fs, double f_comb, double f_offset, int N, int sample_format, int num_sms,
                                int64_t n_rows, pcal_tiling* out) {
    if (!out || num_sms <= 0 || n_rows <= 0) return PCAL_EINVAL;
    pcal_plan tmp;
    memset(static_cast<void*>(&tmp), 0, sizeof(tmp));
    int rc = pcal_plan_geometry(fs, f_comb, f_offset, N, sample_format, &tmp.g);
    if (rc != PCAL_OK) return rc;
    tmp.num_sms = num_sms;
    BulkTiling t;
    if (bulk_tiling(&tmp, n_rows, &t) != 0) return PCAL_EINVAL;
    out->cols_total = t.cols_total;
    out->col_width = t.col_width;
    out->col_groups = t.col_groups;
    out->replicas = t.replicas;
    out->box_rows = t.box_rows;
    out->stages = t.stages;
    out->row_groups = t.row_groups;
    out->rows_per_cta = t.rows_per_cta;
    out->total_boxes = t.total_boxes;
    out->static_boxes = t.static_boxes;
    out->max_boxes = t.max_boxes;
    out->upper_planes = t.upper_planes;
    out->threads = t.threads;
    out->smem_bytes = (int64_t)t.smem_bytes;
    return PCAL_OK;
}
