// Internal declarations of libpcal (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pcal.h"

// 2-bit bins are accumulated as one 64-bit word per bin holding three 21-bit
// fields:  bits 0..20 = sum of l bits, 21..41 = sum of h bits, 42..62 = sum
// of (h AND l).  Together with the known number of samples per bin these give
// the exact counts of all four codes.  The host spills the packed words into
// three wide 64-bit arrays before any field could reach 2^21.
#define PCAL_F21_MASK 0x1FFFFFull
#define PCAL_F21_LIMIT ((1ll << 21) - 1)

// Device-side error flags (bitwise OR into pcal_plan::d_err).
#define PCAL_DERR_FULL_WAIT 1u   // a consumer gave up waiting for a tile
#define PCAL_DERR_EMPTY_WAIT 2u  // the producer gave up waiting for a slot
#define PCAL_DERR_DRAIN_WAIT 4u  // a CTA gave up draining its copies
#define PCAL_DERR_SCHED 8u       // the box counter was not in this launch's epoch

// Tile plan of the bulk kernel for a given plan and row count (host only).
struct BulkTiling {
    int cols_total;    // words per row
    int col_width;     // words per column group (tile width)
    int col_groups;    // G_c
    int replicas;      // consumer threads per column
    int box_rows;      // rows per TMA box (stage)
    int stages;        // pipeline depth
    int64_t row_groups;      // G_r: CTAs per column group
    int64_t rows_per_cta;    // the most rows one CTA can fold (max_boxes * box_rows)
    int total_boxes;         // boxes per column group
    int static_boxes;        // boxes each CTA takes without the shared counter
    int max_boxes;           // cap per CTA
    int chunk;               // boxes per grab from the shared counter
    int upper_planes;  // 2-bit: bit planes above the Harley-Seal tree
    int threads;       // consumer threads + 1 producer warp
    int merge_stride;  // words between rows of the end-of-tile merge area
    size_t smem_bytes;
};

// Encoded tensor maps of recent bulk inputs, so that repeated calls on the
// same buffers skip the host-side encode.
struct BulkMapEntry {
    const void* ptr;
    int64_t rows;
    BulkTiling tiling;
    CUtensorMap map;
};
constexpr int kBulkMapCache = 16;
// SMs the bulk fold leaves free (on GPUs with at least 64 SMs) for the
// one-cluster finalize that overlaps it.
constexpr int kFinalizeReserveSms = 16;
constexpr int kSchedCounters = 8192;  // dynamic box counters (one per column group) + 1

// Where a plan's bulk launch with epoch e starts reading, published by the
// host in ring slot e % kHintRing (pinned, mapped) when it enqueues that
// launch.  The launch before it loads the slot when it starts and, once its
// CTAs have grabbed all their work, pulls the first rows of every row group
// into L2 while it winds down, so the next launch's first copies hit L2
// instead of waiting for HBM.  Only a hint: a prefetch changes no result.
// Each word carries the launch's 16-bit tag (hint_tag) in its top bits and
// is read with one 64-bit load, so a record that is being rewritten shows
// mismatched tags and is skipped.
constexpr int kHintRing = 4096;
struct PrefetchHint {
    unsigned long long rows;    // tag << 48 | rows of the launch
    unsigned long long base;    // tag << 48 | device address of row 0 >> 4 (rows are contiguous)
    unsigned long long groups;  // tag << 48 | row groups << 32 | rows between their first boxes << 16 | rows to pull
};
__host__ __device__ inline unsigned long long hint_tag(unsigned long long epoch) { return epoch % 65535ull + 1ull; }

// Float32 bulk folds write per-tile partial sums into one of kPartSlots
// slots; the finalize adds the pending slots to the bins as it reads them,
// and a reduce kernel adds them when the slots run out or the host reads the
// bins, so consecutive folds (and a fold and its finalize) follow each other
// with no kernel in between.
constexpr int kPartSlots = 4;
struct PartSlot {
    const float2* base;  // [row_groups][cols_total]
    int64_t row_groups;
    int64_t k_a;         // bin of column 0
};

struct pcal_plan {
    pcal_geometry g;
    double levels[4];
    int device;
    int num_sms;
    // stream state
    cudaStream_t last_stream;
    int64_t n_abs;        // samples accumulated since creation
    int64_t period_start; // absolute index of the first sample of this period
    int64_t since_spill;  // 2-bit: samples added since the last spill
    bool spilled;         // 2-bit: the wide arrays hold counts of this period
    // device state
    // Bins, in two sets: accumulates add into set `cur`; a finalize drains
    // set cur and switches cur, so the next period's folds never wait for it.
    int cur;
    unsigned long long* d_acc2;   // 2-bit packed counts [2][L]
    unsigned long long* d_wide2;  // 2-bit spilled counts [2][3][L]
    long long* d_acc8;            // int8 sums [2][L]
    float2* d_accf;               // float32 sums as double-float (hi, lo) [2][L]
    float2* d_partf;              // float32 per-tile partial sums: kPartSlots slots of partf_cap float2
    size_t partf_cap;             // capacity of one slot in float2
    PartSlot pending[kPartSlots]; // slots written by folds and not yet added into the bins
    int n_pending;
    int part_next;                // slot of the next float32 fold
    double2* d_tw;                // exp(-j 2 pi m / L), m < L
    float2* d_twN;                // exp(-j 2 pi m / N), m < N (FP32)
    double2* d_P;                 // folded rotated bins P[b], b < N (scratch)
    double2* d_T;                 // tone phasors (scratch before products)
    double* d_res;                // results, 5N+3 doubles, then the post-processing, N+2 doubles
    unsigned int* d_ticket;       // [0] fold ticket, [1] dft ticket
    unsigned int* d_err;          // device error flags
    unsigned long long* d_sched;  // bulk kernel box counters [kSchedCounters]: (epoch << 32) | boxes
    unsigned int bulk_epoch;      // launches of the bulk kernel (epoch of its counters)
    PrefetchHint* h_hint;         // [kHintRing] pinned, mapped: the bulk launches' read starts
    PrefetchHint* d_hint;         // the same ring as the kernels address it
    // host
    double* h_res;                // pinned copy of d_res
    double* h_ring[2];            // pinned results of pcal_finalize_async (5N+3 values, then the error word)
    cudaEvent_t ring_ev[2];       // ring slot i filled
    int64_t ring_count;           // pcal_finalize_async calls
    void* h_stage[2];             // pinned staging for pcal_accumulate_host
    void* d_stage[2];             // device staging for pcal_accumulate_host
    size_t stage_bytes;
    cudaEvent_t stage_ev[2];      // fold of staging buffer i finished
    cudaEvent_t copied_ev[2];     // copy into staging buffer i finished
    cudaStream_t copy_stream;     // H2D copies of pcal_accumulate_host
    bool results_valid;
    pcal_stats stats;
    BulkMapEntry map_cache[kBulkMapCache];
    int map_next;
};

// The bin set that accumulates currently add into.
inline unsigned long long* cur_acc2(const pcal_plan* p) { return p->d_acc2 + p->cur * p->g.L; }
inline unsigned long long* cur_wide2(const pcal_plan* p) { return p->d_wide2 + p->cur * 3 * p->g.L; }
inline long long* cur_acc8(const pcal_plan* p) { return p->d_acc8 + p->cur * p->g.L; }
inline float2* cur_accf(const pcal_plan* p) { return p->d_accf + p->cur * p->g.L; }

// ---- launchers (return a cudaError_t of the launch) -------------------------
cudaError_t launch_init_twiddles(pcal_plan* p, cudaStream_t s);
cudaError_t launch_ragged(pcal_plan* p, const uint8_t* d_bytes, int64_t n_samples, int64_t k0, cudaStream_t s);
cudaError_t launch_spill2(pcal_plan* p, cudaStream_t s);
cudaError_t launch_export_bins(pcal_plan* p, void* d_out, cudaStream_t s);
cudaError_t launch_finalize(pcal_plan* p, cudaStream_t s);
// Add a float32 plan's pending partial slots into its bins (one reduce launch; none when nothing is pending).
cudaError_t flush_partials(pcal_plan* p, cudaStream_t s);

// Bulk fold of whole rows of row_samples samples starting at a 16-byte
// aligned device address whose first sample has phase k_a = n mod L.
// Returns cudaSuccess and sets *launched = the number of kernels launched,
// or an error.  Rows must be >= 1.
cudaError_t launch_bulk(pcal_plan* p, const void* d_rows, int64_t n_rows, int64_t k_a, cudaStream_t s,
                        int* launched);

int bulk_tiling(const pcal_plan* p, int64_t n_rows, BulkTiling* t);

// ---- batches (pcal_batch_*) ------------------------------------------------------

// One channel of a batch in device memory: its constants, its bins and its
// running sample index.  The kernels advance the index themselves, so a
// captured step can be replayed without the host.
struct BatchChan {
    int fmt;              // PCAL_2BIT or PCAL_I8
    int spw;              // samples per 32-bit word (16 or 4)
    int N;
    int L;
    int64_t so;           // rotator index step per sample: f_offset/g (mod L)
    int cols_total;       // words per bulk row
    int col_width;        // words per column group (the TMA box width)
    int col_groups;
    int64_t row_samples;  // samples per bulk row (a multiple of L)
    unsigned long long* zero2;  // 2-bit: L zero words (the packed fields of the single-plan layout)
    unsigned long long* wide2;  // 2-bit: [3][L] sums of l, h and (h AND l)
    long long* acc8;            // int8: [L] sums
    const double2* tw;          // exp(-j 2 pi m / L), m < L
    const float2* twN;          // exp(-j 2 pi m / N), m < N
    double* res;                // 5N+3 results, then N+2 post-processing values
    double lev0, c_l, c_h, c_hl;
    double two_pi_fc;
    double fs;
    long long n_abs;            // samples accumulated since creation
    long long period_start;     // absolute index of the current period's first sample
    float2* Pslot;              // batched-DFT finalize: this channel's row of P [N]
    float2* Tslot;              // ... and of the tones [N]
};

// One (region, column group) of one call's bulk rows.
struct BatchSeg {
    long long box_start;  // first box in the call's box sequence
    int n_boxes;
    int ch;
    int map;              // tensor map of its region
    int col0;             // first word column of the group
    int tx_bytes;         // bytes one box delivers
    int pad;
    long long head;       // samples of the channel in this call before its first bulk row
};

// A ragged run (head or tail) of one accumulate call.
struct BatchPiece {
    const uint8_t* ptr;   // its first byte
    long long n;          // samples
    long long off;        // offset of its first sample within the call
    int ch;
    int pad;
};

cudaError_t prepare_batch_finalize();
// Finalize of a long-period plan: acc = [lanes][N] double-float bin sums.
cudaError_t launch_rot_finalize(const float4* acc, int lanes, int N, double fs, double fc, int64_t M,
                                const float2* twN, double* res, cudaStream_t s);
// Finalize channels list[i] (or i when list is null), i < n, with one cluster each.
// split: stop every channel after P (its P slot) for the batched DFT, which
// launch_batch_products then finishes.
cudaError_t launch_batch_finalize(BatchChan* d_ch, int n, int max_n, const int* d_list, cudaStream_t s,
                                  int split = 0);
cudaError_t launch_batch_products(BatchChan* d_ch, int n_ch, int max_n, cudaStream_t s);
struct pcal_dft;
// The batched tone DFT of dft_tc.cu (err: device error word, or null for the
// DFT object's own).
cudaError_t launch_dft(pcal_dft* d, const float2* P, int64_t C, float2* T, cudaStream_t s,
                       unsigned int* err = nullptr);
// Operand workspace of launch_dft for up to C channels (allocates).
cudaError_t dft_reserve(pcal_dft* d, int64_t C);

// ---- host side of the batched fold (shared by pcal_batch_* and the server) ----

#include <vector>

// A contiguous run of one channel's samples in device memory.
struct BatchRegion {
    int ch;
    const uint8_t* ptr;
    int64_t n;    // samples
    int64_t off;  // samples of this channel earlier in the same call
};

// Launch shape of the persistent fold for one schedule.
struct BatchShape {
    int wpr, replicas, box_rows, stages, merge_stride, threads, grid, run_boxes, static_pct, min_chunk;
    uint32_t stage_stride;
    size_t smem;
};

// Device descriptors of one call: tensor maps, segments, pieces, samples per
// channel, and the channels to finalize.
struct BatchCallDesc {
    std::vector<uint8_t> blob;  // host image of the device buffer
    size_t off_maps, off_segs, off_pieces, off_n, off_list;
    int n_segs, n_pieces, n_list;
    long long total_boxes;
};

int batch_shape(const pcal_schedule& sc, int cw_max, int num_sms, BatchShape* s);
int batch_build(const BatchChan* h_ch, int n_ch, const std::vector<BatchRegion>& regions, const BatchShape& sh,
                const std::vector<int>& fin_list, BatchCallDesc* out);
cudaError_t batch_launch_fold(const BatchCallDesc& d, void* d_desc, BatchChan* d_ch, int n_ch,
                              unsigned long long* d_ctr, const BatchShape& sh, unsigned int* d_err, cudaStream_t s,
                              int* launches);
cudaError_t batch_prepare_fold();
cudaError_t batch_launch_tables(BatchChan& C, const pcal_geometry& g, cudaStream_t s);
void batch_fill_chan(BatchChan& C, const pcal_geometry& g, double f_comb, const pcal_schedule& sched);
size_t batch_chan_bytes(const pcal_geometry& g);
void batch_place_chan(BatchChan& C, const pcal_geometry& g, uint8_t* base);
