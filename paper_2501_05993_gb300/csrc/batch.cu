// Batched extraction (pcal_batch_*): many channels of mixed sample format,
// sample rate, comb offset, period L and length, folded by ONE persistent
// launch and finalized by one launch with a thread-block cluster per channel.
//
// Work list.  Every channel's call is split like a single-plan call: a
// ragged head up to its first 16-byte boundary, whole rows of row_samples
// samples (a multiple of L, so word c of every row feeds fixed bins), and a
// ragged tail.  The rows of each (channel, column group) form a segment; the
// segments' boxes (box_rows rows of one column group) are numbered one after
// the other into a single box sequence.  Each CTA of the persistent kernel
// takes a contiguous static share of that sequence and then grabs shrinking
// chunks of the rest from one counter (guided self-scheduling), so SMs that
// stream faster take more.
//
// Runs.  A CTA counts in registers while consecutive boxes stay in one
// segment (and below 65,535 rows, which keeps the per-position counts of a
// flush below 2^16); when the segment changes the producer closes the run
// with one marker per consumer group, the CTA merges its replicas and adds
// its counts to that channel's bins with global atomics, and the pipeline
// continues with the next segment.  2-bit sums go to three 64-bit arrays per
// channel (no field can overflow), int8 sums to one.
//
// Graphs.  Every per-call quantity that changes between steps lives on the
// device (each channel's running sample index is advanced by a kernel), so
// a step captured into a CUDA graph is replayed unchanged.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cudaTypedefs.h>

#include "bitplane.cuh"
#include "internal.cuh"
#include "ptx.cuh"

namespace {

using namespace pcal_ptx;

constexpr int kMaxBlock = 512;           // consumer warps + producer warp (<= 128 registers)
constexpr int kSmemBudget = 220 * 1024;  // dynamic shared memory per CTA
constexpr int kRunRows = 65535;          // rows per run (per-position counts < 2^16)
constexpr int kU = 11;                   // upper bit planes: up to 2^16 - 1 rows per thread
constexpr int kSlots = 4;                // descriptor buffers in flight
constexpr int64_t kPieceBytes = 8192;    // ragged runs are cut into pieces of at most this many bytes

struct BatchFoldArgs {
    const CUtensorMap* maps;  // per channel (128-byte entries in device memory)
    const BatchSeg* segs;
    int n_segs;
    BatchChan* ch;
    long long total_boxes;
    long long static_boxes;  // per CTA
    long long pool_start;    // first box handed out by the counter
    int min_chunk;
    // [0] boxes of the pool handed out, [1] pieces handed out, [2] CTAs done;
    // zero at launch, and the last CTA zeroes them again for the next call
    unsigned long long* ctr;
    const BatchPiece* pieces;  // heads and tails of the call's regions
    int n_pieces;
    int n_ch;
    const long long* n_call;  // samples of each channel in the call
    int box_rows;
    int stages;
    int wpr;
    int replicas;
    int merge_stride;
    int run_boxes;
    uint32_t stage_stride;
    unsigned int* err;
};

// 2-bit per-thread counters (see bitplane.cuh).
struct Acc2 {
    uint32_t w1 = 0, w2 = 0, w4 = 0, w8 = 0, w16 = 0, wu[kU];
    uint32_t d1 = 0, d2 = 0, d4 = 0, d8 = 0, du[kU];
    __device__ Acc2() {
#pragma unroll
        for (int u = 0; u < kU; ++u) wu[u] = du[u] = 0;
    }
    __device__ __forceinline__ void add32(const uint32_t (&x)[32]) {
        pcal_bits::add32<kU>(x, w1, w2, w4, w8, w16, wu, d1, d2, d4, d8, du);
    }
};

__device__ int seg_of(const BatchFoldArgs& a, long long g, int hint) {
    if (hint >= 0 && g >= a.segs[hint].box_start && g < a.segs[hint].box_start + a.segs[hint].n_boxes) return hint;
    int lo = 0, hi = a.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].box_start <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// A chunk of the pool: max(min_chunk, remaining / (2 * CTAs)) boxes.
// Returns its first box, -1 when the pool is empty, -2 on failure.
__device__ long long grab_pool(const BatchFoldArgs& a, int* take_out) {
    const long long pool = a.total_boxes - a.pool_start;
    unsigned long long cur = atomicAdd(a.ctr, 0ull);
    for (int i = 0; i < 4096; ++i) {
        const long long taken = (long long)cur;
        if (taken >= pool) return -1;
        long long take = (pool - taken) / (2LL * gridDim.x);
        if (take < a.min_chunk) take = a.min_chunk;
        if (take > pool - taken) take = pool - taken;
        const unsigned long long prev = atomicCAS(a.ctr, cur, cur + (unsigned long long)take);
        if (prev == cur) {
            *take_out = (int)take;
            return a.pool_start + taken;
        }
        cur = prev;
    }
    atomicOr(a.err, PCAL_DERR_SCHED);
    return -2;
}

// One ragged piece (a head or tail run of a region) by all threads of a CTA:
// 2-bit codes add to the three wide sums of their bin, int8 samples to the
// int8 sum.
__device__ void fold_piece(const BatchPiece& P, BatchChan* ch, int tid, int nthreads) {
    const BatchChan& C = ch[P.ch];
    const long long L = C.L;
    const long long k0 = (C.n_abs + P.off) % L;
    if (C.fmt == PCAL_2BIT) {
        unsigned long long* w = C.wide2;
        const long long nb = P.n / 4;
        for (long long i = tid; i < nb; i += nthreads) {
            const uint32_t b = P.ptr[i];
            if (b == 0) continue;
            long long k = (k0 + 4 * i) % L;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t c = (b >> (2 * j)) & 3u;
                if (c & 1u) atomicAdd(&w[k], 1ull);
                if (c & 2u) atomicAdd(&w[L + k], 1ull);
                if (c == 3u) atomicAdd(&w[2 * L + k], 1ull);
                if (++k == L) k = 0;
            }
        }
    } else {
        const int8_t* x = reinterpret_cast<const int8_t*>(P.ptr);
        for (long long i = tid; i < P.n; i += nthreads) {
            const int v = x[i];
            if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&C.acc8[(k0 + i) % L]), (unsigned long long)(long long)v);
        }
    }
}

// Threads: `replicas` groups of `wpr` consumer warps, then one producer warp
// (lane 0 works).  Box j of the CTA (data or marker) lives in stage
// j % stages and belongs to group j % replicas; stages is a multiple of
// replicas, so every stage belongs to one group, which waits for its uses in
// order.  A marker (s_hdr = 1) ends the group's part of the current run.
// After the boxes each CTA takes ragged pieces from a counter; the last CTA
// to finish moves every channel's running index past the call and zeroes the
// counters.  Launched as a programmatic dependent of the preceding kernel:
// every thread waits for it before its first global access.
__global__ void __launch_bounds__(kMaxBlock, 1) batch_fold_kernel(const BatchFoldArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x;
    const int group_threads = a.wpr * 32;
    const int n_cons = a.wpr * a.replicas * 32;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)a.stages * a.stage_stride);
    uint64_t* empty = full + a.stages;
    __shared__ int s_hdr[8];
    __shared__ int s_failed;
    __shared__ int s_next_seg;
    __shared__ int s_last_fill[8];  // per stage: index of its last TMA fill, or -1
    __shared__ int s_fill_open[8];  // per stage: that fill is the stage's latest phase
    __shared__ int s_piece;
    __shared__ int s_last;

    if (tid == 0) {
        s_failed = 0;
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], group_threads);
            s_last_fill[s] = -1;
            s_fill_open[s] = 0;
        }
        fence_barrier_init();
    }
    // the preceding kernel (a finalize or a fold of the same channels) has
    // completed and its bins, indices and counters are visible
    grid_dependency_wait();
    allow_dependents();
    const bool producer = tid == n_cons;
    const bool cons = tid < n_cons;
    const int q = tid / group_threads;
    const int col = tid % group_threads;

    // producer state, kept across runs; the samples are read once, so their
    // L2 lines go first (the bins and tables the finalize reuses stay)
    const uint64_t policy = producer ? l2_policy_evict_first() : 0ull;
    long long st_pos = (long long)blockIdx.x * a.static_boxes;
    long long st_end = st_pos + a.static_boxes;
    if (st_end > a.pool_start) st_end = a.pool_start;
    long long ck_pos = 0, ck_end = 0;
    long long pending = -1;
    int pj = 0;
    auto next_box = [&]() -> long long {
        if (st_pos < st_end) return st_pos++;
        if (ck_pos < ck_end) return ck_pos++;
        int take = 0;
        const long long g = grab_pool(a, &take);
        if (g < 0) return g;
        ck_pos = g + 1;
        ck_end = g + take;
        return g;
    };
    auto stage_free = [&](int jj) -> bool {
        const int s = jj % a.stages;
        const uint32_t use = jj / a.stages;
        if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
            atomicOr(a.err, PCAL_DERR_EMPTY_WAIT);
            return false;
        }
        return true;
    };
    __syncthreads();
    if (producer) {
        pending = next_box();
        if (pending < -1) s_failed = 1;
        s_next_seg = pending >= 0 ? seg_of(a, pending, -1) : -1;
    }
    int cj = q;  // this consumer group's next box index
    __syncthreads();
    int cur = s_failed ? -1 : s_next_seg;
    while (cur >= 0) {
        const BatchSeg seg = a.segs[cur];
        const int fmt = a.ch[seg.ch].fmt;
        const int cw = seg.tx_bytes / (a.box_rows * 4);
        const bool active = cons && col < cw;
        Acc2 acc2;
        int s8[4] = {0, 0, 0, 0};
        if (producer) {
            tensormap_acquire(&a.maps[seg.map]);
            int run = 0, next = -1;
            bool ok = true;
            for (;;) {
                if (pending == -1) pending = next_box();
                if (pending < -1) {
                    ok = false;
                    break;
                }
                if (pending < 0) break;
                const int sg = seg_of(a, pending, cur);
                if (sg != cur || run == a.run_boxes) {
                    next = sg;
                    break;
                }
                if (!stage_free(pj)) {
                    ok = false;
                    break;
                }
                const int st = pj % a.stages;
                s_hdr[st] = 0;
                mbar_arrive_expect_tx(&full[st], (uint32_t)seg.tx_bytes);
                tma_load_2d_hint(smem + (size_t)st * a.stage_stride, &a.maps[seg.map], seg.col0,
                                 (int)(pending - seg.box_start) * a.box_rows, &full[st], policy);
                s_last_fill[st] = pj;
                s_fill_open[st] = 1;
                ++pj;
                ++run;
                pending = -1;
            }
            // one marker per group closes the run
            for (int i = 0; ok && i < a.replicas; ++i) {
                if (!stage_free(pj)) {
                    ok = false;
                    break;
                }
                const int st = pj % a.stages;
                s_hdr[st] = 1;
                s_fill_open[st] = 0;
                mbar_arrive(&full[st]);
                ++pj;
            }
            if (!ok) s_failed = 1;
            s_next_seg = ok ? next : -1;
        } else if (cons) {
            for (;; cj += a.replicas) {
                const int st = cj % a.stages;
                const uint32_t use = cj / a.stages;
                if (!mbar_wait(&full[st], use & 1)) {
                    atomicOr(a.err, PCAL_DERR_FULL_WAIT);
                    s_failed = 1;
                    break;
                }
                if (s_hdr[st] != 0) {
                    mbar_arrive(&empty[st]);
                    cj += a.replicas;
                    break;
                }
                const uint32_t* p = reinterpret_cast<const uint32_t*>(smem + (size_t)st * a.stage_stride) + col;
                if (fmt == PCAL_2BIT) {
                    for (int b = 0; b < a.box_rows; b += 32) {
                        uint32_t x[32];
                        if (active) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) x[i] = p[i * cw];
                        }
                        p += 32 * cw;
                        if (b + 32 >= a.box_rows) mbar_arrive(&empty[st]);  // words are in registers
                        if (active) acc2.add32(x);
                    }
                } else {
                    if (active) {
#pragma unroll 8
                        for (int i = 0; i < a.box_rows; ++i) {
                            const uint32_t w = p[i * cw];
                            s8[0] = __dp4a((int)w, 0x00000001, s8[0]);
                            s8[1] = __dp4a((int)w, 0x00000100, s8[1]);
                            s8[2] = __dp4a((int)w, 0x00010000, s8[2]);
                            s8[3] = __dp4a((int)w, 0x01000000, s8[3]);
                        }
                    }
                    mbar_arrive(&empty[st]);
                }
            }
        }
        __syncthreads();
        if (s_failed) break;

        // ---- merge the replicas of this run, then add to the channel's bins ----
        // (the stage buffers are idle: every fill landed and was consumed)
        const BatchChan& C = a.ch[seg.ch];
        const long long L = C.L;
        const long long k_a = (C.n_abs + seg.head) % L;
        if (fmt == PCAL_2BIT) {
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
            for (int u = 0; u < kU; ++u) {
                if (5 + u < 16) W[5 + u] = acc2.wu[u];
                if (4 + u < 16) D[4 + u] = acc2.du[u];
            }
            // group 0 gathers the l/h planes W, group 1 the (h AND l) planes
            // D; each transposes its planes into counts
            uint32_t* scratch = reinterpret_cast<uint32_t*>(smem);
            const int rc = a.replicas * cw;
            const int qd = a.replicas > 1 ? 1 : 0;
            if (active) {
                uint32_t* dst = scratch + q * cw + col;
                if (q != 0)
#pragma unroll
                    for (int i = 0; i < 16; ++i) dst[i * rc] = W[i];
                if (q != qd)
#pragma unroll
                    for (int i = 0; i < 16; ++i) dst[(16 + i) * rc] = D[i];
            }
            __syncthreads();
            uint32_t* m = scratch + 32 * rc;  // m[i*S + col], i < 32
            if (active && (q == 0 || q == qd)) {
                for (int o = 0; o < a.replicas; ++o) {
                    if (o == q) continue;
                    const uint32_t* src = scratch + o * cw + col;
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
            const int S = a.merge_stride;
            unsigned long long* wide = C.wide2;
            for (int t = tid; t < cw * 16; t += blockDim.x) {
                const int cl = t >> 4, j = t & 15;
                const int gc = seg.col0 + cl;
                if (gc >= C.cols_total) continue;
                const int pl = 2 * j, ph = 2 * j + 1;  // bit positions of l and h
                const uint32_t sl = (m[(pl & 15) * S + cl] >> (16 * (pl >> 4))) & 0xFFFFu;
                const uint32_t sh = (m[(ph & 15) * S + cl] >> (16 * (ph >> 4))) & 0xFFFFu;
                const uint32_t shl = ((m[(16 + (pl & 15)) * S + cl] >> (16 * (pl >> 4))) & 0xFFFFu) +
                                     ((m[(16 + (ph & 15)) * S + cl] >> (16 * (ph >> 4))) & 0xFFFFu);
                const long long bin = (k_a + 16LL * gc + j) % L;
                if (sl) atomicAdd(&wide[bin], (unsigned long long)sl);
                if (sh) atomicAdd(&wide[L + bin], (unsigned long long)sh);
                if (shl) atomicAdd(&wide[2 * L + bin], (unsigned long long)shl);
            }
        } else {
            int* m = reinterpret_cast<int*>(smem);  // m[j*S + col], j < 4
            const int S = a.merge_stride;
            for (int i = tid; i < 4 * S; i += blockDim.x) m[i] = 0;
            __syncthreads();
            if (active) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (s8[j]) atomicAdd(&m[j * S + col], s8[j]);
            }
            __syncthreads();
            for (int t = tid; t < cw * 4; t += blockDim.x) {
                const int cl = t >> 2, j = t & 3;
                const int gc = seg.col0 + cl;
                const int v = m[j * S + cl];
                if (gc >= C.cols_total || v == 0) continue;
                const long long bin = (k_a + 4LL * gc + j) % L;
                atomicAdd(reinterpret_cast<unsigned long long*>(&C.acc8[bin]), (unsigned long long)(long long)v);
            }
        }
        __syncthreads();
        cur = s_next_seg;
    }
    if (s_failed && producer) {
        // TMA fills whose phase no consumer waited for must land before the
        // CTA exits (its shared memory is then reused)
        for (int s = 0; s < a.stages; ++s)
            if (s_fill_open[s] && s_last_fill[s] >= 0 &&
                !mbar_wait(&full[s], (uint32_t)(s_last_fill[s] / a.stages) & 1))
                atomicOr(a.err, PCAL_DERR_DRAIN_WAIT);
    }

    // ---- ragged pieces, taken one at a time by CTAs whose boxes are done ----
    for (;;) {
        if (tid == 0) s_piece = (int)atomicAdd(&a.ctr[1], 1ull);
        __syncthreads();
        const int pi = s_piece;
        __syncthreads();
        if (pi >= a.n_pieces) break;
        fold_piece(a.pieces[pi], a.ch, tid, blockDim.x);
    }

    // ---- the last CTA advances the indices and zeroes the counters ----
    // (every CTA has read the indices it needs before its ticket)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&a.ctr[2], 1ull) == (unsigned long long)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int c = tid; c < a.n_ch; c += blockDim.x) a.ch[c].n_abs += a.n_call[c];
        if (tid == 0) {
            a.ctr[0] = 0;
            a.ctr[1] = 0;
            a.ctr[2] = 0;
        }
    }
}

__global__ void batch_tables_kernel(double2* tw, int64_t L, float2* twN, int64_t N, int64_t sc) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < L; m += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)L, &s, &c);
        tw[m] = make_double2(c, -s);
        if (m % sc == 0 && m / sc < N) twN[m / sc] = make_float2((float)c, (float)-s);
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

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

// ---- host side ---------------------------------------------------------------------

struct BatchGraph {
    std::vector<const void*> ptrs;
    std::vector<int64_t> n;
    void* d_desc;
    unsigned long long* d_ctr;
    cudaGraphExec_t exec;
};

// Channels of one N that share a batched tone DFT: rows of P and of the
// tones, one per channel, contiguous.
struct DftGroup {
    int N;
    int count;
    pcal_dft* dft;
    float2* dP;
    float2* dT;
};

struct pcal_batch {
    int n;
    int device;
    int num_sms;
    std::vector<pcal_geometry> g;
    std::vector<BatchChan> h_ch;  // host copy of the constant parts
    BatchChan* d_ch;
    void* d_pool;
    std::vector<int64_t> n_abs, period_start;  // host mirrors of the device indices
    int cw_max;
    int max_n;  // largest N of the channels
    pcal_schedule sched;
    // descriptor ring for eager calls
    void* h_slot[kSlots];
    void* d_slot[kSlots];
    size_t slot_cap;
    cudaEvent_t slot_ev[kSlots];
    bool slot_used[kSlots];
    size_t slot_len[kSlots];          // bytes of descriptors the slot holds (0: none)
    cudaStream_t slot_stream[kSlots]; // the stream its copy was enqueued on
    bool slot_reused[kSlots];         // read by a fold enqueued after slot_ev
    int slot_next;
    unsigned long long* d_ctr;
    unsigned int* d_err;
    cudaStream_t last_stream;
    std::vector<BatchGraph> graphs;
    pcal_stats stats;
    int dft_mode;                 // PCAL_DFT_FP32: the DFT inside each channel's cluster
    std::vector<DftGroup> dft;    // tensor-core modes: one group per distinct N
};

int batch_shape(const pcal_schedule& sc, int cw_max, int num_sms, BatchShape* s) {
    BatchShape z{};
    z.box_rows = sc.box_rows;
    z.wpr = (cw_max + 31) / 32;
    int r_max = (kMaxBlock / 32 - 1) / z.wpr;
    if (r_max > 8) r_max = 8;
    if (r_max < 1) r_max = 1;
    const size_t stage = (size_t)z.box_rows * cw_max * 4;
    z.stage_stride = (uint32_t)align_up(stage, 1024);
    z.merge_stride = (cw_max + 31) / 32 * 32 + 2;
    z.replicas = 0;
    for (int rr = r_max; rr >= 1 && z.replicas == 0; --rr) {
        int st = (int)((kSmemBudget - 1024) / z.stage_stride);
        if (sc.stages > 0 && st > sc.stages) st = sc.stages;
        if (st > 8) st = 8;
        st = st / rr * rr;
        if (st < 3 || st < rr) continue;
        const size_t need = std::max((size_t)128 * rr * cw_max + (size_t)128 * z.merge_stride,
                                     (size_t)16 * z.merge_stride);
        if (need > (size_t)st * z.stage_stride) continue;
        z.replicas = rr;
        z.stages = st;
    }
    if (z.replicas == 0) return -1;
    z.threads = (z.wpr * z.replicas + 1) * 32;
    z.smem = (size_t)z.stages * z.stage_stride + 16 * (size_t)z.stages;
    z.grid = sc.ctas > 0 ? sc.ctas : num_sms;
    z.run_boxes = kRunRows / z.box_rows;
    z.static_pct = sc.static_pct;
    z.min_chunk = sc.min_chunk > 0 ? sc.min_chunk : 1;
    *s = z;
    return 0;
}

int batch_build(const BatchChan* h_ch, int n_ch, const std::vector<BatchRegion>& regions, const BatchShape& sh,
                const std::vector<int>& fin_list, BatchCallDesc* out) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return PCAL_ECUDA;
    std::vector<CUtensorMap> maps;
    std::vector<BatchSeg> segs;
    std::vector<BatchPiece> pieces;
    std::vector<long long> ncall(n_ch, 0);
    long long total = 0;
    // a ragged run as pieces of at most kPieceBytes (one CTA folds a piece)
    auto add_run = [&](const uint8_t* p, int64_t n, int64_t off, int ch, int spb) {
        const int64_t step = kPieceBytes * spb;
        for (int64_t o = 0; o < n; o += step)
            pieces.push_back(BatchPiece{p + o / spb, n - o < step ? n - o : step, off + o, ch, 0});
    };
    for (const BatchRegion& rg : regions) {
        if (rg.ch < 0 || rg.ch >= n_ch || rg.n < 0) return PCAL_EINVAL;
        const BatchChan& C = h_ch[rg.ch];
        const int64_t nc = rg.n;
        ncall[rg.ch] += nc;
        if (nc == 0) continue;
        const uint8_t* p = rg.ptr;
        const int spb = C.fmt == PCAL_2BIT ? 4 : 1;  // samples per byte
        const int64_t nbytes = nc / spb;
        int64_t head_bytes = (int64_t)((16 - (reinterpret_cast<uintptr_t>(p) & 15)) & 15);
        if (head_bytes > nbytes) head_bytes = nbytes;
        const int64_t row_bytes = C.row_samples / spb;
        const int64_t rows = (nbytes - head_bytes) / row_bytes;
        if (rows < 1) {
            add_run(p, nc, rg.off, rg.ch, spb);
            continue;
        }
        if (head_bytes > 0) add_run(p, head_bytes * spb, rg.off, rg.ch, spb);
        const uint8_t* body = p + head_bytes;
        CUtensorMap map;
        memset(&map, 0, sizeof(map));
        cuuint64_t dims[2] = {(cuuint64_t)C.cols_total, (cuuint64_t)rows};
        cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
        cuuint32_t box[2] = {(cuuint32_t)C.col_width, (cuuint32_t)sh.box_rows};
        cuuint32_t estr[2] = {1, 1};
        // 64-byte L2 promotion: a box's rows are runs of whole 32-byte sectors
        // whose ends rarely fall on 256-byte lines, and the neighbouring
        // column group of the same rows is folded much later (its boxes sit
        // in another segment), so 256-byte promotion read the boundary lines
        // twice (C3: 1.06x the sample bytes, 2.60 ms per fold; 64 B: 2.40 ms;
        // none: 2.51 ms, smaller DRAM requests)
        CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint8_t*>(body), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_64B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return PCAL_EINVAL;
        const int map_index = (int)maps.size();
        maps.push_back(map);
        const int nbox = (int)((rows + sh.box_rows - 1) / sh.box_rows);
        for (int gc = 0; gc < C.col_groups; ++gc) {
            BatchSeg sg{};
            sg.box_start = total;
            sg.n_boxes = nbox;
            sg.ch = rg.ch;
            sg.map = map_index;
            sg.col0 = gc * C.col_width;
            sg.tx_bytes = sh.box_rows * C.col_width * 4;
            sg.head = rg.off + head_bytes * spb;
            segs.push_back(sg);
            total += nbox;
        }
        const int64_t tail_byte = head_bytes + rows * row_bytes;
        if (tail_byte < nbytes) add_run(p + tail_byte, (nbytes - tail_byte) * spb, rg.off + tail_byte * spb, rg.ch, spb);
    }
    if (total >= (1LL << 31)) return PCAL_ETOOLARGE;
    BatchCallDesc d;
    d.off_maps = 0;
    d.off_segs = align_up(sizeof(CUtensorMap) * maps.size(), 128);
    d.off_pieces = align_up(d.off_segs + sizeof(BatchSeg) * segs.size(), 128);
    d.off_n = align_up(d.off_pieces + sizeof(BatchPiece) * pieces.size(), 128);
    d.off_list = align_up(d.off_n + sizeof(long long) * ncall.size(), 128);
    const size_t bytes = align_up(d.off_list + sizeof(int) * fin_list.size(), 128);
    d.blob.assign(bytes, 0);
    if (!maps.empty()) memcpy(d.blob.data() + d.off_maps, maps.data(), sizeof(CUtensorMap) * maps.size());
    if (!segs.empty()) memcpy(d.blob.data() + d.off_segs, segs.data(), sizeof(BatchSeg) * segs.size());
    if (!pieces.empty()) memcpy(d.blob.data() + d.off_pieces, pieces.data(), sizeof(BatchPiece) * pieces.size());
    memcpy(d.blob.data() + d.off_n, ncall.data(), sizeof(long long) * ncall.size());
    if (!fin_list.empty()) memcpy(d.blob.data() + d.off_list, fin_list.data(), sizeof(int) * fin_list.size());
    d.n_segs = (int)segs.size();
    d.n_pieces = (int)pieces.size();
    d.n_list = (int)fin_list.size();
    d.total_boxes = total;
    *out = std::move(d);
    return PCAL_OK;
}

cudaError_t batch_launch_fold(const BatchCallDesc& d, void* d_desc, BatchChan* d_ch, int n_ch,
                              unsigned long long* d_ctr, const BatchShape& sh, unsigned int* d_err, cudaStream_t s,
                              int* launches) {
    uint8_t* base = static_cast<uint8_t*>(d_desc);
    *launches = 0;
    if (d.total_boxes == 0 && d.n_pieces == 0) return cudaSuccess;  // no samples in the call
    BatchFoldArgs a{};
    a.maps = reinterpret_cast<const CUtensorMap*>(base + d.off_maps);
    a.segs = reinterpret_cast<const BatchSeg*>(base + d.off_segs);
    a.n_segs = d.n_segs;
    a.ch = d_ch;
    a.total_boxes = d.total_boxes;
    long long grid = sh.grid;
    const long long work = d.total_boxes > d.n_pieces ? d.total_boxes : d.n_pieces;
    if (grid > work) grid = work;
    a.static_boxes = (long long)((double)sh.static_pct / 100.0 * (double)d.total_boxes / (double)grid);
    a.pool_start = a.static_boxes * grid;
    a.min_chunk = sh.min_chunk;
    a.ctr = d_ctr;
    a.pieces = reinterpret_cast<const BatchPiece*>(base + d.off_pieces);
    a.n_pieces = d.n_pieces;
    a.n_ch = n_ch;
    a.n_call = reinterpret_cast<const long long*>(base + d.off_n);
    a.box_rows = sh.box_rows;
    a.stages = sh.stages;
    a.wpr = sh.wpr;
    a.replicas = sh.replicas;
    a.merge_stride = sh.merge_stride;
    a.run_boxes = sh.run_boxes;
    a.stage_stride = sh.stage_stride;
    a.err = d_err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(sh.threads);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, batch_fold_kernel, a);
    if (e == cudaSuccess) *launches = 1;
    return e;
}

cudaError_t batch_prepare_fold() {
    return cudaFuncSetAttribute(batch_fold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
}

cudaError_t batch_launch_tables(BatchChan& C, const pcal_geometry& g, cudaStream_t s) {
    int grid = (int)((g.L + 255) / 256);
    if (grid > 1024) grid = 1024;
    batch_tables_kernel<<<grid, 256, 0, s>>>(const_cast<double2*>(C.tw), g.L, const_cast<float2*>(C.twN), g.N,
                                             g.step_comb);
    return cudaGetLastError();
}

// Fill the constant part of a channel's device record (pointers excluded).
int sched_bucket(int fmt, int cols_total) {
    const int cls = cols_total <= 256 ? 0 : cols_total <= 1024 ? 1 : cols_total <= 4096 ? 2 : 3;
    return (fmt == PCAL_I8 ? 4 : 0) + cls;
}

int chan_col_cap(const pcal_schedule& sc, int fmt, int cols_total) {
    const int b = sc.col_cap_bucket[sched_bucket(fmt, cols_total)];
    return b > 0 ? b : sc.col_cap;
}

// Column groups of a channel's rows for a width cap: as few groups as the cap
// allows, of equal width rounded up to 8 words.
void chan_cut(BatchChan& C, int cap) {
    int gc = (C.cols_total + cap - 1) / cap;
    int cw = (C.cols_total + gc - 1) / gc;
    cw = (cw + 7) / 8 * 8;
    if (cw > cap) cw = cap;
    C.col_groups = (C.cols_total + cw - 1) / cw;
    C.col_width = cw;
}

void batch_fill_chan(BatchChan& C, const pcal_geometry& g, double f_comb, const pcal_schedule& sc) {
    memset(static_cast<void*>(&C), 0, sizeof(C));
    C.fmt = g.format;
    C.spw = g.samples_per_byte_x4;
    C.N = (int)g.N;
    C.L = (int)g.L;
    C.so = g.step_offset;
    C.row_samples = g.row_samples;
    C.cols_total = (int)(g.row_samples / C.spw);
    chan_cut(C, chan_col_cap(sc, C.fmt, C.cols_total));
    const double lv[4] = {-3.3359, -1.0, 1.0, 3.3359};
    C.lev0 = g.format == PCAL_2BIT ? lv[0] : 0.0;
    C.c_l = g.format == PCAL_2BIT ? lv[1] - lv[0] : 0.0;
    C.c_h = g.format == PCAL_2BIT ? lv[2] - lv[0] : 0.0;
    C.c_hl = g.format == PCAL_2BIT ? lv[3] - lv[2] - lv[1] + lv[0] : 0.0;
    C.two_pi_fc = 6.283185307179586476925 * f_comb;
    C.fs = (double)g.fs;
}

// Device bytes of one channel's bins, tables and results (each part 256-byte aligned).
size_t batch_chan_bytes(const pcal_geometry& g) {
    const size_t L = (size_t)g.L, N = (size_t)g.N;
    size_t n = 0;
    if (g.format == PCAL_2BIT) n += align_up(8 * L, 256) + align_up(24 * L, 256);
    if (g.format == PCAL_I8) n += align_up(8 * L, 256);
    n += align_up(16 * L, 256) + align_up(8 * N, 256) + align_up(8 * (6 * N + 5), 256);
    return n;
}

// Point a channel's record into `base` (batch_chan_bytes(g) bytes, 256-aligned).
void batch_place_chan(BatchChan& C, const pcal_geometry& g, uint8_t* base) {
    const size_t L = (size_t)g.L, N = (size_t)g.N;
    size_t o = 0;
    if (g.format == PCAL_2BIT) {
        C.zero2 = reinterpret_cast<unsigned long long*>(base + o);
        o += align_up(8 * L, 256);
        C.wide2 = reinterpret_cast<unsigned long long*>(base + o);
        o += align_up(24 * L, 256);
    }
    if (g.format == PCAL_I8) {
        C.acc8 = reinterpret_cast<long long*>(base + o);
        o += align_up(8 * L, 256);
    }
    C.tw = reinterpret_cast<double2*>(base + o);
    o += align_up(16 * L, 256);
    C.twN = reinterpret_cast<float2*>(base + o);
    o += align_up(8 * N, 256);
    C.res = reinterpret_cast<double*>(base + o);
}

namespace {

int shape_for(const pcal_batch* b, BatchShape* s) { return batch_shape(b->sched, b->cw_max, b->num_sms, s); }

// Column groups of every channel under a schedule's caps (the rule of
// batch_fill_chan), and the widest group.
void apply_col_caps(pcal_batch* b, const pcal_schedule& sc) {
    b->cw_max = 8;
    for (BatchChan& C : b->h_ch) {
        chan_cut(C, chan_col_cap(sc, C.fmt, C.cols_total));
        if (C.col_width > b->cw_max) b->cw_max = C.col_width;
    }
}

bool same_caps(const pcal_schedule& x, const pcal_schedule& y) {
    if (x.col_cap != y.col_cap) return false;
    for (int i = 0; i < PCAL_SCHED_BUCKETS; ++i)
        if (x.col_cap_bucket[i] != y.col_cap_bucket[i]) return false;
    return true;
}

int build_call(pcal_batch* b, const void* const* samples, const int64_t* n, const BatchShape& sh,
               BatchCallDesc* out) {
    std::vector<BatchRegion> regions;
    for (int c = 0; c < b->n; ++c)
        regions.push_back(BatchRegion{c, static_cast<const uint8_t*>(samples[c]), n[c], 0});
    return batch_build(b->h_ch.data(), b->n, regions, sh, std::vector<int>(), out);
}

cudaError_t launch_call(pcal_batch* b, const BatchCallDesc& d, void* d_desc, unsigned long long* d_ctr,
                        const BatchShape& sh, cudaStream_t s) {
    int launches = 0;
    const cudaError_t e = batch_launch_fold(d, d_desc, b->d_ch, b->n, d_ctr, sh, b->d_err, s, &launches);
    b->stats.kernel_launches += launches;
    if (d.total_boxes > 0) b->stats.bulk_launches += 1;
    return e;
}

}  // namespace

extern "C" int pcal_batch_create(const pcal_channel_desc* channels, int n_channels, pcal_batch** out) {
    if (!out) return PCAL_EINVAL;
    *out = nullptr;
    if (!channels || n_channels <= 0 || n_channels > PCAL_MAX_BATCH) return PCAL_EINVAL;
    pcal_batch* b = new pcal_batch();
    b->n = n_channels;
    b->g.resize(n_channels);
    b->h_ch.resize(n_channels);
    b->n_abs.assign(n_channels, 0);
    b->period_start.assign(n_channels, 0);
    b->sched = pcal_schedule{0, 32, 0, 90, 4, 224, {}};
    size_t pool = 0;
    std::vector<size_t> off(n_channels);
    for (int c = 0; c < n_channels; ++c) {
        const pcal_channel_desc& d = channels[c];
        if (d.sample_format != PCAL_2BIT && d.sample_format != PCAL_I8) {
            delete b;
            return PCAL_EINVAL;
        }
        int rc = pcal_plan_geometry(d.fs, d.f_comb, d.f_offset, d.N, d.sample_format, &b->g[c]);
        if (rc != PCAL_OK) {
            delete b;
            return rc;
        }
        if (b->g[c].N > PCAL_BATCH_MAX_N) {
            delete b;
            return PCAL_ETOOLARGE;
        }
        off[c] = pool;
        pool += batch_chan_bytes(b->g[c]);
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pool, pool);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return e == cudaErrorMemoryAllocation ? PCAL_ENOMEM : PCAL_ECUDA;
    }
    e = cudaMemset(b->d_pool, 0, pool);
    uint8_t* base = static_cast<uint8_t*>(b->d_pool);
    b->cw_max = 8;
    b->max_n = 1;
    for (int c = 0; c < n_channels && e == cudaSuccess; ++c) {
        BatchChan& C = b->h_ch[c];
        batch_fill_chan(C, b->g[c], channels[c].f_comb, b->sched);
        batch_place_chan(C, b->g[c], base + off[c]);
        if (C.col_width > b->cw_max) b->cw_max = C.col_width;
        if (C.N > b->max_n) b->max_n = C.N;
        e = batch_launch_tables(C, b->g[c], nullptr);
    }
    // function attributes now: a stream capture of a step must not set them
    if (e == cudaSuccess) e = batch_prepare_fold();
    if (e == cudaSuccess) e = prepare_batch_finalize();
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ch, sizeof(BatchChan) * n_channels);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_ch, b->h_ch.data(), sizeof(BatchChan) * n_channels, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctr, 256);
    if (e == cudaSuccess) e = cudaMemset(b->d_ctr, 0, 256);  // each fold leaves its counters zero
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 256);
    b->slot_cap = 0;
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
        b->h_slot[i] = nullptr;
        b->d_slot[i] = nullptr;
        b->slot_used[i] = false;
        b->slot_len[i] = 0;
        b->slot_stream[i] = nullptr;
        b->slot_reused[i] = false;
        e = cudaEventCreateWithFlags(&b->slot_ev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        pcal_batch_destroy(b);
        return PCAL_ECUDA;
    }
    b->last_stream = nullptr;
    *out = b;
    return PCAL_OK;
}

namespace {

void free_dft_groups(pcal_batch* b) {
    for (DftGroup& g : b->dft) {
        pcal_dft_destroy(g.dft);
        cudaFree(g.dP);
        cudaFree(g.dT);
    }
    b->dft.clear();
}

// The finalize of every channel: one cluster per channel with its DFT inside,
// or (tensor-core modes) the clusters up to P, one batched DFT per N, then the
// products.
cudaError_t batch_finalize_all(pcal_batch* b, cudaStream_t s, int* launches) {
    if (b->dft_mode == PCAL_DFT_FP32) {
        *launches = 1;
        return launch_batch_finalize(b->d_ch, b->n, b->max_n, nullptr, s);
    }
    cudaError_t e = launch_batch_finalize(b->d_ch, b->n, b->max_n, nullptr, s, 1);
    for (size_t i = 0; e == cudaSuccess && i < b->dft.size(); ++i)
        e = launch_dft(b->dft[i].dft, b->dft[i].dP, b->dft[i].count, b->dft[i].dT, s, b->d_err);
    if (e == cudaSuccess) e = launch_batch_products(b->d_ch, b->n, b->max_n, s);
    *launches = 2 + (int)b->dft.size();
    return e;
}

}  // namespace

extern "C" int pcal_batch_set_dft(pcal_batch* b, int mode) {
    if (!b) return PCAL_EINVAL;
    if (mode != PCAL_DFT_FP32 && mode != PCAL_DFT_TC_TF32X3 && mode != PCAL_DFT_TC_BF16X6) return PCAL_EINVAL;
    if (mode == b->dft_mode) return PCAL_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return PCAL_ECUDA;
    // captured steps hold the old finalize
    for (BatchGraph& gr : b->graphs) {
        cudaGraphExecDestroy(gr.exec);
        cudaFree(gr.d_desc);
        cudaFree(gr.d_ctr);
    }
    b->graphs.clear();
    free_dft_groups(b);
    for (BatchChan& c : b->h_ch) c.Pslot = c.Tslot = nullptr;
    int rc = PCAL_OK;
    if (mode != PCAL_DFT_FP32) {
        for (int c = 0; c < b->n && rc == PCAL_OK; ++c) {
            DftGroup* g = nullptr;
            for (DftGroup& x : b->dft)
                if (x.N == b->h_ch[c].N) g = &x;
            if (!g) {
                b->dft.push_back(DftGroup{b->h_ch[c].N, 0, nullptr, nullptr, nullptr});
                g = &b->dft.back();
                rc = pcal_dft_create(g->N, mode, &g->dft);
            }
            ++g->count;
        }
        for (DftGroup& g : b->dft) {
            if (rc != PCAL_OK) break;
            const size_t bytes = (size_t)g.count * g.N * sizeof(float2);
            if (cudaMalloc(&g.dP, bytes) != cudaSuccess || cudaMalloc(&g.dT, bytes) != cudaSuccess ||
                dft_reserve(g.dft, g.count) != cudaSuccess)
                rc = PCAL_ENOMEM;
            int row = 0;
            for (BatchChan& c : b->h_ch)
                if (rc == PCAL_OK && c.N == g.N) {
                    c.Pslot = g.dP + (size_t)row * g.N;
                    c.Tslot = g.dT + (size_t)row * g.N;
                    ++row;
                }
        }
    }
    // the device copy of the channels: keep the device-side indices
    if (rc == PCAL_OK) {
        std::vector<BatchChan> cur(b->n);
        if (cudaMemcpy(cur.data(), b->d_ch, sizeof(BatchChan) * b->n, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = PCAL_ECUDA;
        for (int c = 0; rc == PCAL_OK && c < b->n; ++c) {
            cur[c].Pslot = b->h_ch[c].Pslot;
            cur[c].Tslot = b->h_ch[c].Tslot;
        }
        if (rc == PCAL_OK &&
            cudaMemcpy(b->d_ch, cur.data(), sizeof(BatchChan) * b->n, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = PCAL_ECUDA;
    }
    if (rc != PCAL_OK) {
        free_dft_groups(b);
        for (BatchChan& c : b->h_ch) c.Pslot = c.Tslot = nullptr;
        b->dft_mode = PCAL_DFT_FP32;
        (void)cudaGetLastError();
        return rc;
    }
    b->dft_mode = mode;
    return PCAL_OK;
}

extern "C" int pcal_batch_destroy(pcal_batch* b) {
    if (!b) return PCAL_OK;
    cudaDeviceSynchronize();
    free_dft_groups(b);
    for (BatchGraph& gr : b->graphs) {
        cudaGraphExecDestroy(gr.exec);
        cudaFree(gr.d_desc);
        cudaFree(gr.d_ctr);
    }
    for (int i = 0; i < kSlots; ++i) {
        if (b->h_slot[i]) cudaFreeHost(b->h_slot[i]);
        if (b->d_slot[i]) cudaFree(b->d_slot[i]);
        if (b->slot_ev[i]) cudaEventDestroy(b->slot_ev[i]);
    }
    cudaFree(b->d_ch);
    cudaFree(b->d_pool);
    cudaFree(b->d_ctr);
    cudaFree(b->d_err);
    (void)cudaGetLastError();
    delete b;
    return PCAL_OK;
}

extern "C" int pcal_batch_get_geometry(const pcal_batch* b, int channel, pcal_geometry* out) {
    if (!b || !out || channel < 0 || channel >= b->n) return PCAL_EINVAL;
    *out = b->g[channel];
    return PCAL_OK;
}

extern "C" int pcal_batch_set_schedule(pcal_batch* b, const pcal_schedule* s) {
    if (!b || !s) return PCAL_EINVAL;
    if (s->ctas < 0 || s->ctas > 64 * b->num_sms || (s->box_rows != 32 && s->box_rows != 64) || s->stages < 0 ||
        s->stages > 8 || s->static_pct < 0 || s->static_pct > 100 || s->min_chunk < 1 || s->min_chunk > 4096 ||
        (s->col_cap != 128 && s->col_cap != 224))
        return PCAL_EINVAL;
    for (int i = 0; i < PCAL_SCHED_BUCKETS; ++i) {
        const int v = s->col_cap_bucket[i];
        if (v != 0 && v != 64 && v != 128 && v != 224) return PCAL_EINVAL;
    }
    const pcal_schedule old = b->sched;
    b->sched = *s;
    if (!same_caps(*s, old)) apply_col_caps(b, *s);
    BatchShape sh;
    if (shape_for(b, &sh) != 0) {
        b->sched = old;
        apply_col_caps(b, old);
        return PCAL_EINVAL;
    }
    return PCAL_OK;
}

extern "C" int pcal_batch_channel_tiling(const pcal_batch* b, int channel, int* bucket, int* col_width,
                                         int* col_groups) {
    if (!b || channel < 0 || channel >= b->n || !bucket || !col_width || !col_groups) return PCAL_EINVAL;
    const BatchChan& C = b->h_ch[channel];
    *bucket = sched_bucket(C.fmt, C.cols_total);
    *col_width = C.col_width;
    *col_groups = C.col_groups;
    return PCAL_OK;
}

extern "C" int pcal_batch_get_schedule(const pcal_batch* b, pcal_schedule* out) {
    if (!b || !out) return PCAL_EINVAL;
    *out = b->sched;
    return PCAL_OK;
}

extern "C" int pcal_batch_accumulate(pcal_batch* b, const void* const* samples, const int64_t* n, void* stream) {
    if (!b || !samples || !n) return PCAL_EINVAL;
    for (int c = 0; c < b->n; ++c) {
        if (n[c] < 0 || (n[c] > 0 && !samples[c])) return PCAL_EINVAL;
        if (b->h_ch[c].fmt == PCAL_2BIT && n[c] % 4 != 0) return PCAL_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchShape sh;
    if (shape_for(b, &sh) != 0) return PCAL_EINVAL;
    BatchCallDesc d;
    int rc = build_call(b, samples, n, sh, &d);
    if (rc != PCAL_OK) return rc;
    // A call that repeats the descriptors of an earlier call on the same
    // stream (same buffers and lengths) reads that call's slot again: no
    // copy, and no stream operation between the previous kernel and the
    // fold, which then starts as its programmatic dependent.
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kSlots; ++k) {
        if (b->slot_len[k] != d.blob.size() || b->slot_stream[k] != s ||
            memcmp(b->h_slot[k], d.blob.data(), d.blob.size()) != 0)
            continue;
        e = launch_call(b, d, b->d_slot[k], b->d_ctr, sh, s);
        if (e != cudaSuccess) return PCAL_ECUDA;
        b->slot_reused[k] = true;
        b->last_stream = s;
        for (int c = 0; c < b->n; ++c) {
            b->n_abs[c] += n[c];
            b->stats.n_abs += n[c];
            b->stats.bytes_folded += b->h_ch[c].fmt == PCAL_2BIT ? n[c] / 4 : n[c];
        }
        return PCAL_OK;
    }
    // otherwise a slot whose previous readers have finished
    auto drain_slot = [&](int k) -> cudaError_t {
        if (!b->slot_used[k]) return cudaSuccess;
        const cudaError_t r = b->slot_reused[k] ? cudaStreamSynchronize(b->slot_stream[k])
                                                : cudaEventSynchronize(b->slot_ev[k]);
        b->slot_reused[k] = false;
        return r;
    };
    const int i = b->slot_next;
    b->slot_next = (i + 1) % kSlots;
    e = drain_slot(i);
    b->slot_len[i] = 0;
    if (e == cudaSuccess && d.blob.size() > b->slot_cap) {
        for (int k = 0; k < kSlots; ++k) {
            if (e == cudaSuccess) e = drain_slot(k);
            if (b->h_slot[k]) cudaFreeHost(b->h_slot[k]);
            if (b->d_slot[k]) cudaFree(b->d_slot[k]);
            b->h_slot[k] = b->d_slot[k] = nullptr;
            b->slot_used[k] = false;
            b->slot_len[k] = 0;
        }
        const size_t cap = align_up(d.blob.size() * 2, 4096);
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
            e = cudaMallocHost(&b->h_slot[k], cap);
            if (e == cudaSuccess) e = cudaMalloc(&b->d_slot[k], cap);
        }
        if (e != cudaSuccess) return PCAL_ENOMEM;
        b->slot_cap = cap;
    }
    if (e != cudaSuccess) return PCAL_ECUDA;
    memcpy(b->h_slot[i], d.blob.data(), d.blob.size());
    e = cudaMemcpyAsync(b->d_slot[i], b->h_slot[i], d.blob.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_call(b, d, b->d_slot[i], b->d_ctr, sh, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->slot_ev[i], s);
    if (e != cudaSuccess) return PCAL_ECUDA;
    b->slot_used[i] = true;
    b->slot_len[i] = d.blob.size();
    b->slot_stream[i] = s;
    b->last_stream = s;
    for (int c = 0; c < b->n; ++c) {
        b->n_abs[c] += n[c];
        b->stats.n_abs += n[c];
        b->stats.bytes_folded += b->h_ch[c].fmt == PCAL_2BIT ? n[c] / 4 : n[c];
    }
    return PCAL_OK;
}

extern "C" int pcal_batch_finalize_device(pcal_batch* b, void* stream) {
    if (!b) return PCAL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int launches = 0;
    cudaError_t e = batch_finalize_all(b, s, &launches);
    if (e != cudaSuccess) return PCAL_ECUDA;
    b->stats.kernel_launches += launches;
    b->last_stream = s;
    for (int c = 0; c < b->n; ++c) b->period_start[c] = b->n_abs[c];
    return PCAL_OK;
}

// One whole step (accumulate + finalize) of a fixed set of inputs, captured
// into a CUDA graph on its first use and replayed afterwards.
extern "C" int pcal_batch_step_graph(pcal_batch* b, const void* const* samples, const int64_t* n, void* stream) {
    if (!b || !samples || !n) return PCAL_EINVAL;
    for (int c = 0; c < b->n; ++c) {
        if (n[c] < 0 || (n[c] > 0 && !samples[c])) return PCAL_EINVAL;
        if (b->h_ch[c].fmt == PCAL_2BIT && n[c] % 4 != 0) return PCAL_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchGraph* hit = nullptr;
    for (BatchGraph& gr : b->graphs) {
        bool same = true;
        for (int c = 0; c < b->n && same; ++c) same = gr.ptrs[c] == samples[c] && gr.n[c] == n[c];
        if (same) hit = &gr;
    }
    if (!hit) {
        BatchShape sh;
        if (shape_for(b, &sh) != 0) return PCAL_EINVAL;
        BatchCallDesc d;
        int rc = build_call(b, samples, n, sh, &d);
        if (rc != PCAL_OK) return rc;
        BatchGraph gr;
        gr.ptrs.assign(samples, samples + b->n);
        gr.n.assign(n, n + b->n);
        gr.d_desc = nullptr;
        gr.d_ctr = nullptr;
        gr.exec = nullptr;
        cudaError_t e = cudaMalloc(&gr.d_desc, d.blob.size());
        if (e == cudaSuccess) e = cudaMalloc(&gr.d_ctr, 256);
        if (e == cudaSuccess) e = cudaMemset(gr.d_ctr, 0, 256);  // each fold leaves its counters zero
        if (e == cudaSuccess) e = cudaMemcpy(gr.d_desc, d.blob.data(), d.blob.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaStream_t cap = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const pcal_stats keep = b->stats;
            cudaError_t el = launch_call(b, d, gr.d_desc, gr.d_ctr, sh, cap);
            int fl = 0;
            if (el == cudaSuccess) el = batch_finalize_all(b, cap, &fl);
            b->stats = keep;
            e = cudaStreamEndCapture(cap, &graph);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gr.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFree(gr.d_desc);
            cudaFree(gr.d_ctr);
            return PCAL_ECUDA;
        }
        b->graphs.push_back(gr);
        hit = &b->graphs.back();
    }
    if (cudaGraphLaunch(hit->exec, s) != cudaSuccess) return PCAL_ECUDA;
    b->last_stream = s;
    for (int c = 0; c < b->n; ++c) {
        b->n_abs[c] += n[c];
        b->period_start[c] = b->n_abs[c];
    }
    return PCAL_OK;
}

namespace {

int sync_and_check(pcal_batch* b) {
    cudaError_t e = b->last_stream ? cudaStreamSynchronize(b->last_stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return PCAL_ECUDA;
    unsigned int err = 0;
    if (cudaMemcpy(&err, b->d_err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return PCAL_ECUDA;
    return err ? PCAL_ETIMEOUT : PCAL_OK;
}

}  // namespace

extern "C" int pcal_batch_read_results(pcal_batch* b, int channel, double* phasors, double* amp, double* phase,
                                       double* unwrapped, double* td, double* sigma) {
    if (!b || channel < 0 || channel >= b->n) return PCAL_EINVAL;
    int rc = sync_and_check(b);
    if (rc != PCAL_OK) return rc;
    const int64_t N = b->g[channel].N;
    std::vector<double> r(5 * N + 3);
    if (cudaMemcpy(r.data(), b->h_ch[channel].res, sizeof(double) * r.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PCAL_ECUDA;
    if (phasors) memcpy(phasors, r.data(), sizeof(double) * 2 * N);
    if (amp) memcpy(amp, r.data() + 2 * N, sizeof(double) * N);
    if (phase) memcpy(phase, r.data() + 3 * N, sizeof(double) * N);
    if (unwrapped) memcpy(unwrapped, r.data() + 4 * N, sizeof(double) * N);
    if (td) *td = r[5 * N];
    if (sigma) *sigma = r[5 * N + 1];
    return PCAL_OK;
}

extern "C" int pcal_batch_read_post(pcal_batch* b, int channel, double* td_peak, double* peak_bin,
                                    double* bandpass_phase) {
    if (!b || channel < 0 || channel >= b->n) return PCAL_EINVAL;
    int rc = sync_and_check(b);
    if (rc != PCAL_OK) return rc;
    const int64_t N = b->g[channel].N;
    std::vector<double> r(N + 2);
    if (cudaMemcpy(r.data(), b->h_ch[channel].res + 5 * N + 3, sizeof(double) * r.size(), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return PCAL_ECUDA;
    if (td_peak) *td_peak = r[0];
    if (peak_bin) *peak_bin = r[1];
    if (bandpass_phase) memcpy(bandpass_phase, r.data() + 2, sizeof(double) * N);
    return PCAL_OK;
}

extern "C" int pcal_batch_result_device(const pcal_batch* b, int channel, const double** out) {
    if (!b || !out || channel < 0 || channel >= b->n) return PCAL_EINVAL;
    *out = b->h_ch[channel].res;
    return PCAL_OK;
}

extern "C" int pcal_batch_get_bins(pcal_batch* b, int channel, int64_t* host_out) {
    if (!b || !host_out || channel < 0 || channel >= b->n) return PCAL_EINVAL;
    int rc = sync_and_check(b);
    if (rc != PCAL_OK) return rc;
    const BatchChan& C = b->h_ch[channel];
    const int64_t L = C.L;
    if (C.fmt == PCAL_I8) {
        return cudaMemcpy(host_out, C.acc8, sizeof(int64_t) * L, cudaMemcpyDeviceToHost) == cudaSuccess ? PCAL_OK
                                                                                                     : PCAL_ECUDA;
    }
    std::vector<unsigned long long> w(3 * L);
    if (cudaMemcpy(w.data(), C.wide2, sizeof(unsigned long long) * 3 * L, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PCAL_ECUDA;
    const int64_t n_tot = b->n_abs[channel] - b->period_start[channel];
    const int64_t q = n_tot / L, rem = n_tot % L, a0 = b->period_start[channel] % L;
    for (int64_t k = 0; k < L; ++k) {
        const int64_t sl = (int64_t)w[k], sh = (int64_t)w[L + k], shl = (int64_t)w[2 * L + k];
        const int64_t cnt = q + (((k - a0) % L + L) % L < rem ? 1 : 0);
        host_out[4 * k + 3] = shl;
        host_out[4 * k + 2] = sh - shl;
        host_out[4 * k + 1] = sl - shl;
        host_out[4 * k + 0] = cnt - sl - sh + shl;
    }
    return PCAL_OK;
}

extern "C" int pcal_batch_get_stats(const pcal_batch* b, pcal_stats* out) {
    if (!b || !out) return PCAL_EINVAL;
    *out = b->stats;
    return PCAL_OK;
}

// Time each candidate schedule on the caller's inputs (accumulate only) and
// keep the fastest.  The bins must be empty (a period boundary); they are
// emptied again and the running indices restored afterwards.
extern "C" int pcal_batch_autotune(pcal_batch* b, const void* const* samples, const int64_t* n, void* stream,
                                   pcal_schedule* chosen) {
    if (!b || !samples || !n) return PCAL_EINVAL;
    for (int c = 0; c < b->n; ++c)
        if (b->n_abs[c] != b->period_start[c]) return PCAL_EBUSY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<pcal_schedule> cand;
    // (on the 64-channel mixed batch the larger smallest-chunks won: 8 -> 64 took a step from 2.86 to 2.74 ms)
    for (int cap : {224, 128})
        for (int rows : {32, 64})
            for (int pct : {85, 95})
                for (int chunk : {8, 32, 64, 128}) cand.push_back(pcal_schedule{0, rows, 0, pct, chunk, cap, {}});
    const pcal_schedule keep = b->sched;
    const int cw_keep = b->cw_max;
    const std::vector<BatchChan> ch_keep = b->h_ch;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = PCAL_OK;
    // time one candidate: `reps` accumulates after one that warms up (ms per accumulate, or < 0)
    auto time_cand = [&](const pcal_schedule& cs, int reps) -> float {
        b->sched = cs;
        apply_col_caps(b, cs);
        BatchShape sh;
        if (shape_for(b, &sh) != 0) return -1.f;
        float ms = 0.f;
        for (int rep = 0; rep <= reps && rc == PCAL_OK; ++rep) {
            cudaEventRecord(e0, s);
            rc = pcal_batch_accumulate(b, samples, n, stream);
            cudaEventRecord(e1, s);
            if (rc == PCAL_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = PCAL_ECUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;  // the first run warms up
        }
        return rc == PCAL_OK ? ms / reps : -1.f;
    };
    // pass 1, batch-wide: every candidate briefly, then the four fastest again with more runs
    std::vector<std::pair<float, int>> score;
    for (int i = 0; i < (int)cand.size() && rc == PCAL_OK; ++i) {
        const float ms = time_cand(cand[i], 2);
        if (ms >= 0.f) score.emplace_back(ms, i);
    }
    std::sort(score.begin(), score.end());
    float best = 1e30f;
    pcal_schedule best_s = keep;
    for (int k = 0; k < (int)score.size() && k < 4 && rc == PCAL_OK; ++k) {
        const float ms = time_cand(cand[score[k].second], 6);
        if (ms >= 0.f && ms < best) {
            best = ms;
            best_s = cand[score[k].second];
        }
    }
    // a change is kept when it is faster by more than the timing noise
    auto try_cand = [&](const pcal_schedule& cs) {
        const float ms = time_cand(cs, 6);
        if (ms >= 0.f && ms < best * 0.995f) {
            best = ms;
            best_s = cs;
        }
    };
    // pass 2: the CTA count of the one launch (SMs left idle can shorten the tail of a
    // launch whose work does not divide evenly)
    if (rc == PCAL_OK && best < 1e30f) {
        for (int less : {8, 16}) {
            if (b->num_sms - less < 1 || rc != PCAL_OK) continue;
            pcal_schedule cs = best_s;
            cs.ctas = b->num_sms - less;
            try_cand(cs);
        }
    }
    // pass 3: per (format, row width) bucket the batch occupies, the bucket's own width cap
    bool occupied[PCAL_SCHED_BUCKETS] = {};
    for (const BatchChan& C : ch_keep) occupied[sched_bucket(C.fmt, C.cols_total)] = true;
    for (int bk = 0; bk < PCAL_SCHED_BUCKETS && rc == PCAL_OK && best < 1e30f; ++bk) {
        if (!occupied[bk]) continue;
        const pcal_schedule base = best_s;
        for (int cap : {64, 128, 224}) {
            const int now = base.col_cap_bucket[bk] > 0 ? base.col_cap_bucket[bk] : base.col_cap;
            if (rc != PCAL_OK || cap == now) continue;  // the cap the bucket already has
            pcal_schedule cs = base;
            cs.col_cap_bucket[bk] = cap;
            try_cand(cs);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore: empty bins, indices back to the period boundary
    cudaError_t e = cudaStreamSynchronize(s);
    for (int c = 0; c < b->n && e == cudaSuccess; ++c) {
        b->n_abs[c] = b->period_start[c];
        const BatchChan& C = b->h_ch[c];
        if (C.wide2) e = cudaMemset(C.wide2, 0, sizeof(unsigned long long) * 3 * C.L);
        if (e == cudaSuccess && C.acc8) e = cudaMemset(C.acc8, 0, sizeof(long long) * C.L);
    }
    b->h_ch = ch_keep;
    b->cw_max = cw_keep;
    b->sched = keep;
    for (int c = 0; c < b->n; ++c) {
        b->h_ch[c].n_abs = b->n_abs[c];
        b->h_ch[c].period_start = b->period_start[c];
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_ch, b->h_ch.data(), sizeof(BatchChan) * b->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return PCAL_ECUDA;
    if (rc != PCAL_OK) return rc;
    rc = pcal_batch_set_schedule(b, &best_s);
    if (rc == PCAL_OK && chosen) *chosen = best_s;
    return rc;
}
