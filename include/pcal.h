/*
 * pcal.h -- C ABI of libpcal, a GB300 (sm_103a) implementation of fast
 * multi-tone phase-calibration (PCal) signal extraction.
 *
 * Method (paper Sec. 2): the baseband stream x[n] carries a comb of N tones
 * at frequencies i*f_comb + f_offset (Eq. 1).  Rotating by exp(-j*w_offset*n)
 * (Eq. 3) and folding modulo N_bins = fs/f_comb (Eq. 2) turns the comb into a
 * pulse P whose DFT gives one complex phasor per tone.  The rotator repeats
 * every N_rotator = fs/gcd(fs, f_offset) samples (Eq. 4), so the whole
 * rotate-then-fold is periodic in L = lcm(N_bins, N_rotator) = fs/gcd(fs,
 * f_comb, f_offset).  libpcal therefore folds FIRST: it keeps exact integer
 * per-bin statistics of the raw samples over n mod L (2-bit: per-(bin, code)
 * counts; int8: integer sums; float32: compensated FP32 sums), and rotates,
 * folds and transforms only the L bins when a result is asked for.
 *
 * Conventions shared by every entry point:
 *   - Every call returns PCAL_OK (0) or a negative PCAL_E* code; nothing
 *     aborts or throws across this boundary.  pcal_strerror() names a code.
 *   - "device" pointers are CUDA global-memory addresses of the current
 *     device; "host" pointers are ordinary process memory.  The caller owns
 *     every buffer it passes in; the plan owns all of its own device state.
 *   - `stream` is a cudaStream_t passed as an opaque pointer (NULL = the
 *     legacy default stream).  Asynchronous calls only enqueue work.
 *   - Sample index n is ABSOLUTE: it counts every sample accumulated into the
 *     plan since pcal_plan_create, across calls and integration periods, so
 *     tone phases are referenced to n = 0 of the plan.
 *   - The tone phasor convention is the raw sum
 *         T_i = sum_n x[n] * exp(-j*2*pi*(i*f_comb + f_offset)*n/fs),
 *     i = 0..N-1, forward sign as in Eq. 3, no normalisation.
 *   - A plan is not thread safe: one host thread drives it at a time.
 */
#ifndef PCAL_H
#define PCAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PCAL_OK 0
#define PCAL_EINVAL (-1)    /* an argument is out of range or inconsistent  */
#define PCAL_ENOMEM (-2)    /* a device or pinned-host allocation failed    */
#define PCAL_ECUDA (-3)     /* a CUDA runtime call failed                   */
#define PCAL_EBUSY (-4)     /* the plan cannot take this call right now     */
#define PCAL_ETOOLARGE (-5) /* L (or N) exceeds the library's limits        */
#define PCAL_ETIMEOUT (-6)  /* a bounded device-side wait gave up           */

/* ---- sample formats ---------------------------------------------------- */
#define PCAL_F32 0  /* real IEEE float32, one sample per 4 bytes            */
#define PCAL_I8 1   /* two's-complement int8, one sample per byte           */
#define PCAL_2BIT 2 /* 2-bit codes c = (h<<1)|l, four samples per byte,
                       sample j of a byte in bits 2j..2j+1 (LSB first);
                       decoded through a 4-entry level table               */

/* Library limits. */
#define PCAL_MAX_L 1048576   /* largest combined period L accepted          */
#define PCAL_MAX_N 8192      /* largest number of tones N accepted          */

/*
 * Plan geometry (Eq. 4 and N = fs/f_comb from the text after Eq. 1).
 * Filled by pcal_plan_geometry; all frequencies in integral Hz.
 */
typedef struct {
    int64_t fs, f_comb, f_offset; /* Hz                                      */
    int64_t N;                    /* tones = N_bins = fs / f_comb            */
    int64_t N_rot;                /* fs / gcd(fs, f_offset)       (Eq. 4)    */
    int64_t L;                    /* lcm(N, N_rot) = fs / gcd(fs, fc, fo)    */
    int64_t step_comb;            /* f_comb / gcd: tone spacing in 2*pi/L    */
    int64_t step_offset;          /* f_offset / gcd: offset in 2*pi/L        */
    int32_t format;               /* PCAL_F32, PCAL_I8 or PCAL_2BIT          */
    int32_t samples_per_byte_x4;  /* 1 (f32), 4 (i8) or 16 (2-bit): samples
                                     per 4-byte word                         */
    int64_t row_samples;          /* super-period row of the bulk kernel:
                                     a multiple of L and of the samples in
                                     16 bytes, at least 256 bytes long       */
} pcal_geometry;

/*
 * pcal_plan_geometry -- validate a plan and compute its periods, on the host
 * only (no CUDA call).  fs, f_comb, f_offset must be finite, integral Hz with
 * fs > 0, f_comb > 0, 0 <= f_offset < f_comb and f_comb dividing fs; N must
 * equal fs/f_comb.  Returns PCAL_EINVAL for a bad argument and
 * PCAL_ETOOLARGE when L > PCAL_MAX_L or N > PCAL_MAX_N.  `out` (host) is
 * written only on success.
 */
int pcal_plan_geometry(double fs, double f_comb, double f_offset, int N, int sample_format, pcal_geometry* out);

typedef struct pcal_plan pcal_plan;

/*
 * pcal_plan_create -- make a plan on the current CUDA device (paper Sec. 2,
 * Eq. 1-4).  Validates exactly like pcal_plan_geometry, then allocates the
 * plan's device bins (zeroed), its FP64 twiddle table exp(-j*2*pi*m/L),
 * m < L, and a pinned host result buffer.  On success *out (host) receives
 * the plan, which the caller releases with pcal_plan_destroy.  The 2-bit
 * level table defaults to {-3.3359, -1, +1, +3.3359}.  Errors: PCAL_EINVAL,
 * PCAL_ETOOLARGE, PCAL_ENOMEM, PCAL_ECUDA; on error nothing is allocated.
 */
int pcal_plan_create(double fs, double f_comb, double f_offset, int N, int sample_format, pcal_plan** out);

/* pcal_plan_destroy -- synchronise the plan's last stream and free every
 * resource of the plan.  NULL is accepted. */
int pcal_plan_destroy(pcal_plan* plan);

/* pcal_plan_get_geometry -- copy the plan's geometry to host memory. */
int pcal_plan_get_geometry(const pcal_plan* plan, pcal_geometry* out);

/*
 * pcal_plan_set_levels -- set the values of the 2-bit codes 0..3 (host array
 * of 4 finite doubles).  Takes effect at the next finalize; the integer
 * counts are independent of the levels.  PCAL_EINVAL for non-2-bit plans.
 */
int pcal_plan_set_levels(pcal_plan* plan, const double levels[4]);

/*
 * pcal_accumulate -- fold n samples into the plan's bins (Eq. 2 and Eq. 3
 * combined through the period L of Eq. 4; the fold-first form of Sec. 4.1's
 * long-accumulator remark).
 *   samples: DEVICE pointer to n samples in the plan's format, any alignment
 *            (2-bit: n must be a multiple of 4, i.e. whole bytes).  The caller
 *            keeps it valid until `stream` has passed this call.
 *   n:       number of samples, >= 0; 0 is a no-op.
 *   stream:  cudaStream_t the work is enqueued on; no host synchronisation.
 * The samples continue the plan's absolute index.  Errors: PCAL_EINVAL (bad
 * n or NULL pointer with n > 0), PCAL_ECUDA (launch failure).
 */
int pcal_accumulate(pcal_plan* plan, const void* samples, int64_t n, void* stream);

/*
 * pcal_accumulate_host -- as pcal_accumulate, from a HOST buffer.  The
 * samples are copied to the device through the plan's staging buffers in
 * chunks that overlap copy and fold; the call returns when the host buffer
 * may be reused (the fold itself may still be running on `stream`).  Pinned
 * host memory gives the full copy bandwidth.
 */
int pcal_accumulate_host(pcal_plan* plan, const void* host_samples, int64_t n, void* stream);

/*
 * pcal_accumulate_host_async -- as pcal_accumulate_host, but returns as soon
 * as the copies and folds are queued: the host buffer must stay unchanged
 * until `stream` has passed this call's folds (a later synchronising call on
 * the plan, a stream synchronisation, or pcal_read_async_results of a period
 * finalized after it).  Lets a host loop queue the next period's copies
 * while the link is still busy with this one.
 */
int pcal_accumulate_host_async(pcal_plan* plan, const void* host_samples, int64_t n, void* stream);

/*
 * pcal_finalize_device -- end the current integration period on `stream`
 * (NULL = the stream of the last accumulate):  decode the bins, rotate each
 * of the L bins by exp(-j*2*pi*f_offset*k/fs) in FP64 (Eq. 3), fold them to
 * N bins (Eq. 2), take the N-point DFT (DFT(P), Sec. 2), then amplitude
 * 2|T_i|/M, phase arg(T_i)+pi/2 (the sin model of Eq. 1), the phase unwrapped
 * along the comb and the instrumental delay t_d as the |T|^2-weighted
 * least-squares slope of phase versus tone frequency (phi_i = 2*pi*f_i*t_d,
 * Eq. 1).  Results stay in the plan's device result buffer (see
 * pcal_result_device); the bins are reset to zero for the next period and
 * the absolute sample index keeps counting.  Asynchronous.
 */
int pcal_finalize_device(pcal_plan* plan, void* stream);

/*
 * pcal_finalize -- pcal_finalize_device on the stream of the last
 * accumulate, then wait for it and copy the N raw phasors T_i to
 * phasors_out (HOST, 2*N doubles, re/im interleaved).  phasors_out may be
 * NULL when only the products below are wanted.
 */
int pcal_finalize(pcal_plan* plan, double* phasors_out);

/*
 * pcal_read_results -- wait for the last finalize and copy its results to
 * host arrays (any of them may be NULL): phasors 2*N (re/im), amp N, phase N
 * (wrapped to [-pi, pi)), unwrapped N, and td_s / sigma_td_s (seconds).
 */
int pcal_read_results(pcal_plan* plan, double* phasors, double* amp, double* phase, double* unwrapped,
                      double* td_s, double* sigma_td_s);

/*
 * Pipelined results.  pcal_finalize_async -- pcal_finalize_device on
 * `stream`, then an asynchronous copy of the period's results (the 5N+3
 * values of pcal_read_results and the device error bits) into a pinned ring
 * of two slots; returns at once.  pcal_read_async_results -- wait for the
 * results of the period finalized `age` pcal_finalize_async calls ago (0 =
 * the latest, 1 = the one before; a slot is reused two calls later) and
 * copy them out as pcal_read_results does.  PCAL_EINVAL for an age not held
 * in the ring, PCAL_ETIMEOUT if a bounded device wait of that period gave up.
 */
int pcal_finalize_async(pcal_plan* plan, void* stream);
int pcal_read_async_results(pcal_plan* plan, int age, double* phasors, double* amp, double* phase,
                            double* unwrapped, double* td_s, double* sigma_td_s);

/* pcal_get_delay -- delay and its 1-sigma of the last finalize (host). */
int pcal_get_delay(pcal_plan* plan, double* td_s, double* sigma_td_s);

/*
 * Post-processing of the last finalize (synchronises the plan's stream):
 *   td_peak:  the delay from the time-domain pulse P (the folded, rotated
 *             bins, Eq. 2-3): the largest |P[b]| and the vertex of the parabola
 *             through it and its neighbours (the three-point estimate of Sec. 2);
 *             a delay t_d puts the pulse at b = -t_d*fs (mod N), so
 *             td_peak = -(b + d)/fs wrapped into [-1/(2 f_comb), 1/(2 f_comb)).
 *   peak_bin: b + d, the interpolated pulse position in bins.
 *   bandpass_phase: HOST, N doubles: each tone's unwrapped phase minus the
 *             weighted LS line (the group-delay-corrected bandpass of Sec. 3);
 *             NaN when no fit exists.
 * Any pointer may be NULL.  They live on the device right after the 5N+3
 * doubles of pcal_result_device.
 */
int pcal_read_post(pcal_plan* plan, double* td_peak, double* peak_bin, double* bandpass_phase);

/*
 * pcal_result_device -- device address of the plan's result buffer, laid out
 * as doubles: [0,2N) phasors re/im, [2N,3N) amp, [3N,4N) phase, [4N,5N)
 * unwrapped phase, 5N td, 5N+1 sigma_td, 5N+2 samples integrated.  Owned by
 * the plan; valid until pcal_plan_destroy.
 */
const double* pcal_result_device(const pcal_plan* plan);

/*
 * pcal_get_bins -- synchronise and copy the bins of the CURRENT integration
 * period to host memory, exactly:  2-bit: int64 counts[L][4] of each code
 * per bin; int8: int64 sums[L]; float32: double sums[L] (the compensated
 * FP32 partial sums combined in FP64).  Bin k holds samples with absolute
 * index n = k mod L.
 */
int pcal_get_bins(pcal_plan* plan, void* host_out);

/* Counters of a plan (host). */
typedef struct {
    int64_t n_abs;          /* samples accumulated since plan creation      */
    int64_t n_period;       /* samples in the current integration period    */
    int64_t kernel_launches;/* CUDA kernels this plan has launched          */
    int64_t bulk_launches;  /* of which bulk (TMA bit-plane) fold kernels   */
    int64_t bytes_folded;   /* sample bytes folded on the device            */
} pcal_stats;

/* Copy the plan's counters into *out (host bookkeeping; no CUDA call, no
 * synchronisation).  PCAL_EINVAL for a NULL argument. */
int pcal_get_stats(const pcal_plan* plan, pcal_stats* out);

/*
 * Work split of the bulk fold kernel (host only, no CUDA call), for tests and
 * diagnostics: how `n_rows` rows of `row_samples` samples are tiled over
 * `num_sms` SMs for a plan with these parameters.  PCAL_EINVAL when no tile
 * plan exists (such inputs are folded by the ragged kernel instead).
 */
typedef struct {
    int32_t cols_total, col_width, col_groups, replicas, box_rows, stages;
    int64_t row_groups, rows_per_cta;   /* CTAs per column group; most rows one CTA folds */
    int32_t upper_planes, threads;
    int64_t smem_bytes;
    int32_t total_boxes, static_boxes, max_boxes;  /* per column group; per CTA */
} pcal_tiling;

/* fs, f_comb, f_offset, N, sample_format: as pcal_plan_create; num_sms >= 1;
 * n_rows >= 1 rows of the plan's row_samples (pcal_plan_geometry); *out is
 * written on PCAL_OK. */
int pcal_bulk_tiling(double fs, double f_comb, double f_offset, int N, int sample_format, int num_sms,
                     int64_t n_rows, pcal_tiling* out);

/*
 * pcal_tones_from_counts_noalloc -- the finalize (decode, rotate, fold to N,
 * DFT, products) for callers that cannot allocate GPU memory: code that runs
 * inside a fixed memory pool or arena, a process whose device memory is
 * budgeted up front, or a stream being captured into a CUDA graph (where a
 * cudaMalloc is not allowed).  It creates no plan and calls no cudaMalloc,
 * cudaFree or allocating library routine.  The paper has no counterpart:
 * this is an interface choice of this library.
 *   fs, f_comb, f_offset, N: validated as in pcal_plan_geometry; N must be
 *            at most 1024 (PCAL_ETOOLARGE otherwise).
 *   d_counts: DEVICE, int64 [L][4], the per-(bin, code) counts of a 2-bit
 *            stream as pcal_get_bins returns them (bin k = samples with
 *            absolute index n = k mod L).  Read only.
 *   n_samples: samples the counts cover (the M of the amplitude 2|T|/M).
 *   levels:  HOST, the 4 code values.
 *   d_results: DEVICE, 5N+3 doubles, written with the layout of
 *            pcal_result_device.
 *   stream:  cudaStream_t; the call only enqueues work.
 * Scratch lives in a static device array of about 24.6 KB that every GPU
 * loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.  All
 * calls on a device share the array and it keeps the previous call's
 * contents (the call clears what must start at zero), so calls whose GPU
 * work overlaps -- on different streams or host threads -- race; serialise
 * them.
 */
int pcal_tones_from_counts_noalloc(double fs, double f_comb, double f_offset, int N, const int64_t* d_counts,
                                   int64_t n_samples, const double levels[4], double* d_results, void* stream);

/*
 * ---- Batches: many channels, one persistent fold launch ----------------------
 *
 * A batch holds up to PCAL_MAX_BATCH channels (2-bit or int8 samples), each
 * with its own fs, f_comb, f_offset and N, hence its own period L (Eq. 4).
 * One pcal_batch_accumulate call folds a run of samples of every channel with
 * ONE persistent kernel launch over a work list of all channels' tiles; the
 * same launch folds the ragged heads and tails (pieces of at most 8 KB) and
 * its last CTA advances the channels' sample indices.  A call that repeats
 * the buffers and lengths of an earlier call on the same stream reuses that
 * call's device descriptors without a copy.  pcal_batch_finalize_device
 * turns every channel's bins into its N phasors, amplitude, phase and delay
 * (Sec. 2) with one launch, a thread-block cluster per channel.  The bins
 * are exact integers, so a channel's counts and phasors do not depend on the
 * batch it is folded in or on the schedule.  The paper processes one stream at a
 * time; batching is an interface choice of this library.
 */
#define PCAL_MAX_BATCH 4096   /* channels per batch                           */
#define PCAL_BATCH_MAX_N 1024 /* tones per batched channel                    */

typedef struct {
    double fs, f_comb, f_offset; /* Hz, integral, as for pcal_plan_create     */
    int N;                       /* fs / f_comb                               */
    int sample_format;           /* PCAL_2BIT or PCAL_I8                      */
} pcal_channel_desc;

/* Launch schedule of the persistent fold (pcal_batch_autotune picks one).
 * A channel's tile is a column group of its rows (one row = a whole number of
 * periods L); its width is capped by the channel's bucket -- sample format x
 * row width -- or, where the bucket's cap is 0, by col_cap.  Bucket index =
 * 4 * (format == PCAL_I8) + class, class 0: rows of at most 256 32-bit
 * words, 1: at most 1024, 2: at most 4096, 3: wider.  box_rows, stages and
 * ctas shape the one launch, so they are per batch. */
#define PCAL_SCHED_BUCKETS 8
typedef struct {
    int ctas;        /* CTAs of the fold launch; 0 = one per SM                */
    int box_rows;    /* rows per TMA box: 32 or 64                              */
    int stages;      /* pipeline stages, 0 = as many as fit (at most 8)         */
    int static_pct;  /* percent of the boxes handed out statically (0..100)     */
    int min_chunk;   /* smallest dynamic grab, boxes (1..4096)                  */
    int col_cap;     /* widest column group, 32-bit words: 128 or 224           */
    int col_cap_bucket[PCAL_SCHED_BUCKETS]; /* per bucket: 0 (= col_cap), 64, 128 or 224 */
} pcal_schedule;

typedef struct pcal_batch pcal_batch;

/*
 * Create a batch on the current device: validates every channel as
 * pcal_plan_create does (PCAL_EINVAL for an F32 channel, PCAL_ETOOLARGE for
 * N > PCAL_BATCH_MAX_N), allocates all bins, tables and results in one device
 * allocation the batch owns, and builds the FP64 rotator tables.  Levels of
 * 2-bit channels: {-3.3359, -1, +1, +3.3359}.  Synchronous.
 */
int pcal_batch_create(const pcal_channel_desc* channels, int n_channels, pcal_batch** out);
int pcal_batch_destroy(pcal_batch* batch);
int pcal_batch_get_geometry(const pcal_batch* batch, int channel, pcal_geometry* out);
int pcal_batch_set_schedule(pcal_batch* batch, const pcal_schedule* sched);
/* How the batch finalize runs the tone DFT (the PCAL_DFT_* modes of the
 * batched tone DFT below): PCAL_DFT_FP32 (default) inside each channel's
 * finalize cluster on CUDA cores; PCAL_DFT_TC_TF32X3 / PCAL_DFT_TC_BF16X6 as
 * one tensor-core contraction per distinct N over all channels of that N (the
 * clusters stop at P, then a products kernel finishes every channel).
 * Synchronises the device; drops captured step graphs. */
int pcal_batch_set_dft(pcal_batch* batch, int mode);
int pcal_batch_get_schedule(const pcal_batch* batch, pcal_schedule* out);
/* The tile a channel's rows are cut into under the current schedule (host only): its bucket (the
 * index into col_cap_bucket), the column-group width in 32-bit words and the number of groups. */
int pcal_batch_channel_tiling(const pcal_batch* batch, int channel, int* bucket, int* col_width, int* col_groups);

/*
 * Fold n[c] more samples of every channel c.  samples: HOST array of
 * n_channels DEVICE pointers (any alignment; the caller keeps each buffer
 * valid until the stream passes this call); n: HOST array of sample counts
 * (0 skips a channel; 2-bit counts are multiples of 4).  Samples continue each
 * channel's absolute index.  Asynchronous on `stream` (cudaStream_t).
 */
int pcal_batch_accumulate(pcal_batch* batch, const void* const* samples, const int64_t* n, void* stream);

/* Finalize every channel on `stream` (results stay on the device) and start
 * each channel's next period.  Asynchronous. */
int pcal_batch_finalize_device(pcal_batch* batch, void* stream);

/*
 * pcal_batch_accumulate + pcal_batch_finalize_device as one CUDA graph: the
 * first call with a given set of (samples, n) captures the step, later calls
 * with the same pointers and counts replay it (the buffers' contents may
 * change).  Every per-step quantity lives on the device, so replays continue
 * the channels' sample indices correctly.  Asynchronous.
 */
int pcal_batch_step_graph(pcal_batch* batch, const void* const* samples, const int64_t* n, void* stream);

/* Results of one channel after a finalize (synchronises the batch's last
 * stream; PCAL_ETIMEOUT if a device wait gave up).  Layout and NULL handling
 * as pcal_read_results. */
int pcal_batch_read_results(pcal_batch* batch, int channel, double* phasors, double* amp, double* phase,
                            double* unwrapped, double* td, double* sigma);

/* Post-processing of one channel (pcal_read_post's definitions; synchronises). */
int pcal_batch_read_post(pcal_batch* batch, int channel, double* td_peak, double* peak_bin, double* bandpass_phase);

/* Device address of one channel's result vector (layout of pcal_result_device). */
int pcal_batch_result_device(const pcal_batch* batch, int channel, const double** out);

/* The current period's exact bins of one channel (synchronises): 2-bit:
 * int64 [L][4] per-code counts; int8: int64 [L] sums. */
int pcal_batch_get_bins(pcal_batch* batch, int channel, int64_t* host_out);

/* The batch's counters summed over its channels (n_abs: samples accumulated;
 * n_period is not kept and stays 0): host bookkeeping, no synchronisation.
 * PCAL_EINVAL for a NULL argument. */
int pcal_batch_get_stats(const pcal_batch* batch, pcal_stats* out);

/*
 * Time candidate schedules on these inputs, accumulate only, and keep the
 * fastest; writes it to *chosen when not NULL.  Three passes: the batch-wide
 * choices (column-width cap, box rows, static share, chunk size; the four
 * fastest timed again), then the CTA count (one per SM, or 8 or 16 fewer),
 * then, one bucket at a time for the buckets the batch's channels occupy, the
 * bucket's own column-width cap (64, 128, 224), each kept only when it is
 * faster.  The batch must be at a period boundary (PCAL_EBUSY otherwise); its
 * bins are emptied and its indices restored afterwards.  Synchronous.
 */
int pcal_batch_autotune(pcal_batch* batch, const void* const* samples, const int64_t* n, void* stream,
                        pcal_schedule* chosen);

/*
 * ---- Serving: continuous batching of live streams ----------------------------
 *
 * A server holds up to max_streams live streams (2-bit or int8, each with its
 * own fs, f_comb, f_offset, N).  A stream is admitted when its device memory
 * -- bins, rotator table, results and a ring of ring_s seconds of samples --
 * fits in what remains of hbm_budget_bytes (one device allocation the server
 * owns); otherwise it is queued and admitted as closed streams return memory.
 * Clients submit chunks of host samples; a scheduler thread folds every
 * stream's pending samples with one persistent launch (the batched fold),
 * finalizes each stream once period_s seconds of its samples are folded
 * (Sec. 2), and publishes the results with their latency: from the arrival
 * of the chunk that brought a period's last sample (the time the client
 * stamps on it with pcal_server_submit_many_at, else the return of its
 * submit) to the moment the results are on the host.
 * Work submitted while the GPU is busy joins the next launch (several are in
 * flight).  The paper has no counterpart; serving is an interface choice of
 * this library.  All calls are thread-safe; one client thread per stream.
 */
typedef struct {
    int64_t hbm_budget_bytes; /* device memory for all streams                  */
    int max_streams;          /* streams admitted at once, at most              */
    double period_s;          /* integration period (fs*period_s samples, a multiple of 4) */
    double ring_s;            /* device ring per stream, seconds of samples     */
} pcal_server_config;

typedef struct {
    int32_t stream, n_tones;
    int64_t period;           /* 0, 1, 2, ... for this stream                   */
    int64_t n_samples;        /* samples in the period                          */
    double td_s, sigma_td_s;  /* delay and its 1-sigma                          */
    double latency_s;         /* arrival of the period's last chunk -> results on the host */
    double td_peak_s;         /* delay from the time-domain pulse (pcal_read_post) */
} pcal_server_result;

typedef struct {
    int64_t admitted, queued, active, periods, samples, launches, bytes_h2d;
    int64_t hbm_in_use, hbm_budget;
    double p50_latency_s, p99_latency_s, max_latency_s;
} pcal_server_stats;

typedef struct pcal_server pcal_server;

/* Device bytes a stream takes from the budget (host only, no CUDA call). */
int pcal_server_stream_bytes(const pcal_server_config* config, const pcal_channel_desc* desc, int64_t* out);
/* Create a server on the current device (allocates the whole budget, starts the scheduler thread). */
int pcal_server_create(const pcal_server_config* config, pcal_server** out);
/* Stop the scheduler after the work in flight; free everything.  Unfinished periods are dropped. */
int pcal_server_destroy(pcal_server* server);
/* Open a stream: validated as pcal_batch_create's channels; PCAL_ENOMEM if it could never fit the
 * budget.  *stream_id is valid at once; the stream is admitted now or later (queued). */
int pcal_server_open(pcal_server* server, const pcal_channel_desc* desc, int* stream_id);
/* Copy n samples (HOST memory, pinned for speed; n a multiple of 4 for 2-bit, at most the ring)
 * into the stream's device ring.  Blocks while the stream is queued or its ring is full; returns
 * when the copy is done (the host buffer may then be reused). */
int pcal_server_submit(pcal_server* server, int stream_id, const void* host_samples, int64_t n);
/* One chunk for each of `count` distinct streams, copied together. */
int pcal_server_submit_many(pcal_server* server, int count, const int* stream_ids, const void* const* host_samples,
                            const int64_t* n);
/* As pcal_server_submit_many, with the arrival time of each chunk (arrival_s: HOST, `count` times
 * in seconds of pcal_clock_s; NULL = the submit's return): a period's latency is measured from
 * the arrival of its last chunk, so time the chunk spent waiting for the client, for admission,
 * for ring space and for its copy counts.  PCAL_EINVAL for a NaN time. */
int pcal_server_submit_many_at(pcal_server* server, int count, const int* stream_ids,
                               const void* const* host_samples, const int64_t* n, const double* arrival_s);
/* The library's monotonic clock in seconds (the clock of arrival times and latencies). */
double pcal_clock_s(void);
/* Close a stream: its submitted samples are still folded, a partial period is dropped, then its
 * memory returns to the budget. */
int pcal_server_close(pcal_server* server, int stream_id);
/* Next published result: 1 and *out (and the 2*n_tones phasors, re/im interleaved, into phasors
 * when not NULL; max_tones is its capacity in tones), or 0 when none arrived within timeout_s. */
int pcal_server_poll(pcal_server* server, pcal_server_result* out, double* phasors, int max_tones,
                     double timeout_s);
/* Wait until every submitted sample is folded and every closed stream released. */
int pcal_server_drain(pcal_server* server, double timeout_s);
/* Counters and latency percentiles over all published periods. */
int pcal_server_get_stats(pcal_server* server, pcal_server_stats* out);

/*
 * ---- Precision study: the paper's per-sample rotation in FP32 ----------------
 *
 * pcal_rotfold_* runs the paper's own route for comparison with the fold-first
 * integer path: every sample rotated by exp(-j w_o n) (Eq. 3) and added into
 * bin n mod N (Eq. 2) in FP32, with the rotator from an FP32 table of N_rot
 * entries (Eq. 4) or from the direct-form second-order resonator (Eq. 9), and
 * the FP32 sums plain or Kahan-compensated; then the bins are DFT'd in FP64.
 * Thread (lane, b) sums the samples n = b (mod N) with (n div N) = lane
 * (mod lanes) in sample order, so every FP32 operation has a fixed order; its
 * accumulator persists across calls until the finalize.  int8 or float32
 * samples.  The resonator steps over one thread's samples (N*lanes apart) and
 * is seeded from the exact FP64 phase at each thread's first sample of a call.
 */
#define PCAL_ROT_TABLE 0        /* FP32 rotator table, plain FP32 sums        */
#define PCAL_ROT_TABLE_KAHAN 1  /* FP32 rotator table, Kahan-compensated sums */
#define PCAL_ROT_DFR 2          /* FP32 resonator (Eq. 9), plain FP32 sums    */

typedef struct pcal_rotfold pcal_rotfold;

/* fs, f_comb, f_offset, N: as pcal_plan_create (the same geometry checks);
 * sample_format PCAL_I8 or PCAL_F32; variant one of PCAL_ROT_*; lanes
 * 1..4096 accumulators per bin.  Allocates the device state, which the
 * object owns (PCAL_ENOMEM, PCAL_ECUDA); PCAL_EINVAL for other values. */
int pcal_rotfold_create(double fs, double f_comb, double f_offset, int N, int sample_format, int variant, int lanes,
                        pcal_rotfold** out);
/* Frees the object's device state once its work has finished (NULL: no-op). */
int pcal_rotfold_destroy(pcal_rotfold* r);
/* samples: DEVICE, n samples continuing the absolute index; asynchronous on stream. */
int pcal_rotfold_accumulate(pcal_rotfold* r, const void* samples, int64_t n, void* stream);
/* Lanes added in FP64, N-point DFT in FP64; phasors_out: HOST, 2N doubles (re, im).  Synchronises
 * `stream`, then clears the accumulators (the absolute index keeps counting). */
int pcal_rotfold_finalize(pcal_rotfold* r, double* phasors_out, void* stream);
/* The FP32 accumulators, float [lanes][N][4] = (sum re, sum im, compensation re, compensation im). */
int pcal_rotfold_get_acc(pcal_rotfold* r, float* host_out);

/*
 * ---- Long-period plans: offsets that cannot be folded -----------------------
 *
 * For a comb offset whose combined period L (Eq. 4) is beyond PCAL_MAX_L (a
 * prime offset) or that is not a whole number of hertz, pcal_rotplan_* rotates
 * every sample (Eq. 3) into N bins (Eq. 2) in double-float: per thread a
 * rotator advanced by one complex multiplication per sample and re-seeded
 * every 256 samples from the exact phase frac(n*f_offset/fs) (double-double,
 * FP64 sincospi); then the DFT, the products and the post-processing of the
 * folded path.  fs and f_comb integral Hz, N = fs/f_comb <= PCAL_BATCH_MAX_N,
 * 0 <= f_offset < f_comb any value; f32, int8 or 2-bit samples; at most 2^52
 * samples per plan.  The throughput is arithmetic-bound (several times below
 * the folded path).
 */
typedef struct pcal_rotplan pcal_rotplan;

/* fs, f_comb: integral Hz with N = fs/f_comb (PCAL_EINVAL otherwise),
 * N <= PCAL_BATCH_MAX_N (PCAL_ETOOLARGE); 0 <= f_offset < f_comb, any value;
 * sample_format PCAL_F32, PCAL_I8 or PCAL_2BIT.  Allocates the device state,
 * which the object owns (PCAL_ENOMEM, PCAL_ECUDA). */
int pcal_rotplan_create(double fs, double f_comb, double f_offset, int N, int sample_format, pcal_rotplan** out);
/* Waits for the object's last stream, then frees it (NULL: no-op). */
int pcal_rotplan_destroy(pcal_rotplan* plan);
/* 2-bit decode levels of codes 0..3 (host array, copied), as pcal_plan_set_levels. */
int pcal_rotplan_set_levels(pcal_rotplan* plan, const double levels[4]);
/* samples: DEVICE, n samples continuing the absolute index; asynchronous on stream. */
int pcal_rotplan_accumulate(pcal_rotplan* plan, const void* samples, int64_t n, void* stream);
/* Finalize on `stream` (results stay on the device) and start the next period. */
int pcal_rotplan_finalize_device(pcal_rotplan* plan, void* stream);
/* Results of the last finalize (synchronises; layout as pcal_read_results and pcal_read_post;
 * any pointer may be NULL). */
int pcal_rotplan_read_results(pcal_rotplan* plan, double* phasors, double* amp, double* phase, double* unwrapped,
                              double* td, double* sigma, double* td_peak, double* bandpass_phase);

/*
 * ---- Batched tone DFT -------------------------------------------------------
 *
 * T_i = sum_b P[b] e^{-j 2 pi i b / N} for C channels at once (the DFT of P of
 * Sec. 2, after the L-to-N fold of Eq. 2).  P and T: DEVICE, C x N complex
 * float32 (re, im interleaved, channel-major), owned by the caller; T may not
 * alias P.  Modes:
 *   PCAL_DFT_FP32       CUDA cores, FP32 sums
 *   PCAL_DFT_TC_TF32X3  tensor cores (tcgen05): [Re P | Im P] . W as one real
 *                       C x 2N x 2N contraction, operands split in two TF32
 *                       parts (x = h + l), three products
 *   PCAL_DFT_TC_BF16X6  the same with three BF16 parts (x = h + m + l) and
 *                       the six products of total order <= 2
 * In both tensor-core modes every K chunk (32 values per row) starts a fresh
 * FP32 accumulator in tensor memory, which is added into FP32 registers on
 * CUDA cores (round to nearest) while the next chunk accumulates: the error
 * stays at the level of an FP32 sum.  Errors vs FP64 at C = 4096, N = 1024,
 * max over channels of max|T - T_ref| / max|T_ref|, measured on GB300:
 * FP32 2.8e-6, TF32x3 6.1e-7, BF16x6 4.2e-7.
 * pcal_dft_create builds the weight tiles (2N x 2N, split, in the layout the
 * kernel copies; 32 MB (TF32) or 24 MB (BF16) for N = 1024) once;
 * 1 <= N <= PCAL_BATCH_MAX_N.
 * pcal_dft_execute is asynchronous on `stream`; C <= 65535 * 128.  Its
 * operand workspace grows (cudaMalloc) when C exceeds every earlier call's.
 * pcal_dft_check synchronises and returns PCAL_ETIMEOUT (with the device
 * error bits) if a bounded wait inside the kernel gave up.
 * A tile is 128 channels x 256 output columns; K goes in chunks of 128
 * bytes per row (TF32x3: 32 values) or 64 bytes (BF16x6: 32 values).
 * pcal_dft_weights_host writes weight tile (tile, chunk) of a tensor-core
 * mode into `parts` (HOST, 3 x 256 x B bytes, B = the mode's chunk bytes:
 * part p at byte 256 * B * p; rows = the tile's output columns, at most 256,
 * returned in *rows; the mode's number of parts, 2 or 3, in *n_parts);
 * host-only, for tests of the layout.
 */
#define PCAL_DFT_FP32 0
#define PCAL_DFT_TC_TF32X3 1
#define PCAL_DFT_TC_BF16X6 2
typedef struct pcal_dft pcal_dft;

/* PCAL_EINVAL for N or mode out of range, PCAL_ENOMEM / PCAL_ECUDA when the
 * device state cannot be made; the object owns it. */
int pcal_dft_create(int N, int mode, pcal_dft** out);
/* Synchronises the device and frees the object (NULL: no-op). */
int pcal_dft_destroy(pcal_dft* dft);
/* PCAL_EINVAL for C < 0 or NULL P / T with C > 0; PCAL_ETOOLARGE beyond C
 * limit; C = 0 launches nothing. */
int pcal_dft_execute(pcal_dft* dft, const void* P, int64_t C, void* T, void* stream);
int pcal_dft_check(pcal_dft* dft, unsigned int* flags_out);
/* PCAL_EINVAL for the CUDA-core mode, N out of range, or tile / chunk
 * outside the weight matrix. */
int pcal_dft_weights_host(int N, int mode, int tile, int chunk, void* parts, int* rows, int* n_parts);

/*
 * Failure detection without a fault: one block waits, with the bounded
 * mbarrier wait every TMA-fed kernel uses, on a phase nothing completes, for
 * limit_s seconds (0 < limit_s <= 2), records that it gave up and returns
 * normally.  Returns PCAL_ETIMEOUT with *flags_out = the device error bits
 * (the expected outcome: the context stays usable), PCAL_OK if nothing gave
 * up.  Synchronous; for tests and diagnostics.
 */
int pcal_selftest_wait_timeout(double limit_s, unsigned int* flags_out);

/* Static name of a status code. */
const char* pcal_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* PCAL_H */
