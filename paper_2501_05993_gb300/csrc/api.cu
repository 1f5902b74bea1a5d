// C ABI of libpcal: plan lifetime, accumulate orchestration, finalize and
// result transfer.  Every step of the extraction runs in this library's CUDA
// kernels; the host side only validates, splits work and enqueues.
#include <stdlib.h>
#include <string.h>

#include <new>

#include "internal.cuh"

namespace {

// Inputs shorter than this many bulk rows (or bytes) go through the ragged
// kernel alone: the bulk kernel's fixed cost does not pay off below it.
constexpr int64_t kBulkMinBytes = 1 << 20;
constexpr size_t kStageBytes = 64ull << 20;

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PCAL_OK;
    if (e == cudaErrorMemoryAllocation) return PCAL_ENOMEM;
    return PCAL_ECUDA;
}

void free_plan(pcal_plan* p) {
    if (!p) return;
    cudaFree(p->d_acc2);
    cudaFree(p->d_wide2);
    cudaFree(p->d_acc8);
    cudaFree(p->d_accf);
    cudaFree(p->d_partf);
    cudaFree(p->d_tw);
    cudaFree(p->d_twN);
    cudaFree(p->d_P);
    cudaFree(p->d_T);
    cudaFree(p->d_res);
    cudaFree(p->d_ticket);
    cudaFree(p->d_err);
    cudaFree(p->d_sched);
    for (int i = 0; i < 2; ++i) {
        cudaFree(p->d_stage[i]);
        if (p->stage_ev[i]) cudaEventDestroy(p->stage_ev[i]);
        if (p->copied_ev[i]) cudaEventDestroy(p->copied_ev[i]);
    }
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->h_res) cudaFreeHost(p->h_res);
    for (int i = 0; i < 2; ++i) {
        if (p->h_ring[i]) cudaFreeHost(p->h_ring[i]);
        if (p->ring_ev[i]) cudaEventDestroy(p->ring_ev[i]);
    }
    if (p->h_hint) cudaFreeHost(p->h_hint);
    delete p;
}

template <typename T>
cudaError_t dalloc(T** ptr, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T) + 16);
    if (e == cudaSuccess) e = cudaMemset(*ptr, 0, count * sizeof(T) + 16);
    return e;
}

int64_t bytes_of(const pcal_plan* p, int64_t n) {
    switch (p->g.format) {
        case PCAL_F32: return 4 * n;
        case PCAL_I8: return n;
        default: return n / 4;
    }
}

// Samples in `b` bytes of the plan's format.
int64_t samples_of(const pcal_plan* p, int64_t b) {
    switch (p->g.format) {
        case PCAL_F32: return b / 4;
        case PCAL_I8: return b;
        default: return 4 * b;
    }
}

// Fold one run of samples (n small enough for the packed 2-bit fields).
int accumulate_run(pcal_plan* p, const uint8_t* d, int64_t n, cudaStream_t s) {
    const int64_t L = p->g.L;
    const int64_t k0 = p->n_abs % L;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(d);
    int64_t head = samples_of(p, (int64_t)((16 - addr % 16) % 16));
    if (head > n) head = n;
    const int64_t row = p->g.row_samples;
    int64_t rows = (n - head) / row;
    if (bytes_of(p, rows * row) < kBulkMinBytes) rows = 0;
    BulkTiling probe;
    if (rows > 0 && bulk_tiling(p, rows, &probe) != 0) rows = 0;  // no tile plan: ragged only
    cudaError_t e = cudaSuccess;
    if (rows == 0) {
        e = launch_ragged(p, d, n, k0, s);
    } else {
        if (head > 0) e = launch_ragged(p, d, head, k0, s);
        const uint8_t* body = d + bytes_of(p, head);
        int launched = 0;
        if (e == cudaSuccess) e = launch_bulk(p, body, rows, (k0 + head) % L, s, &launched);
        if (e == cudaSuccess) p->stats.bulk_launches += 1;
        const int64_t done = head + rows * row;
        if (e == cudaSuccess && done < n)
            e = launch_ragged(p, body + bytes_of(p, rows * row), n - done, (k0 + done) % L, s);
    }
    if (e != cudaSuccess) return cuda_status(e);
    p->n_abs += n;
    p->since_spill += n;
    p->stats.bytes_folded += bytes_of(p, n);
    return PCAL_OK;
}

}  // namespace

extern "C" int pcal_plan_create(double fs, double f_comb, double f_offset, int N, int sample_format, pcal_plan** out) {
    if (!out) return PCAL_EINVAL;
    pcal_geometry g;
    int rc = pcal_plan_geometry(fs, f_comb, f_offset, N, sample_format, &g);
    if (rc != PCAL_OK) return rc;
    pcal_plan* p = new (std::nothrow) pcal_plan();
    if (!p) return PCAL_ENOMEM;
    memset(static_cast<void*>(p), 0, sizeof(*p));
    p->g = g;
    const double lv[4] = {-3.3359, -1.0, 1.0, 3.3359};
    memcpy(p->levels, lv, sizeof(lv));
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    const int64_t L = g.L, Nn = g.N;
    if (e == cudaSuccess) {
        if (g.format == PCAL_2BIT) {
            e = dalloc(&p->d_acc2, 2 * L);
            if (e == cudaSuccess) e = dalloc(&p->d_wide2, 2 * 3 * L);
        } else if (g.format == PCAL_I8) {
            e = dalloc(&p->d_acc8, 2 * L);
        } else {
            e = dalloc(&p->d_accf, 2 * L);
        }
    }
    if (e == cudaSuccess) e = dalloc(&p->d_tw, L);
    if (e == cudaSuccess) e = dalloc(&p->d_twN, Nn);
    if (e == cudaSuccess) e = dalloc(&p->d_P, Nn);
    if (e == cudaSuccess) e = dalloc(&p->d_T, Nn);
    if (e == cudaSuccess) e = dalloc(&p->d_res, 6 * Nn + 5);
    if (e == cudaSuccess) e = dalloc(&p->d_ticket, 4);
    if (e == cudaSuccess) e = dalloc(&p->d_err, 4);
    if (e == cudaSuccess) e = dalloc(&p->d_sched, kSchedCounters);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&p->h_res), (6 * Nn + 5) * sizeof(double));
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void**>(&p->h_hint), kHintRing * sizeof(PrefetchHint), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        memset(static_cast<void*>(p->h_hint), 0, kHintRing * sizeof(PrefetchHint));
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&p->d_hint), p->h_hint, 0);
    }
    if (e == cudaSuccess) e = launch_init_twiddles(p, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_status(e);
    }
    p->last_stream = 0;
    *out = p;
    return PCAL_OK;
}

extern "C" int pcal_plan_destroy(pcal_plan* p) {
    if (!p) return PCAL_OK;
    cudaStreamSynchronize(p->last_stream);
    free_plan(p);
    return PCAL_OK;
}

extern "C" int pcal_plan_get_geometry(const pcal_plan* p, pcal_geometry* out) {
    if (!p || !out) return PCAL_EINVAL;
    *out = p->g;
    return PCAL_OK;
}

extern "C" int pcal_plan_set_levels(pcal_plan* p, const double levels[4]) {
    if (!p || !levels || p->g.format != PCAL_2BIT) return PCAL_EINVAL;
    for (int i = 0; i < 4; ++i)
        if (!(levels[i] == levels[i]) || levels[i] > 1e300 || levels[i] < -1e300) return PCAL_EINVAL;
    memcpy(p->levels, levels, sizeof(p->levels));
    return PCAL_OK;
}

extern "C" int pcal_accumulate(pcal_plan* p, const void* samples, int64_t n, void* stream) {
    if (!p || n < 0) return PCAL_EINVAL;
    if (n == 0) return PCAL_OK;
    if (!samples) return PCAL_EINVAL;
    if (p->g.format == PCAL_2BIT && n % 4 != 0) return PCAL_EINVAL;
    if (p->g.format == PCAL_F32 && reinterpret_cast<uintptr_t>(samples) % 4 != 0) return PCAL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->last_stream = s;
    const uint8_t* d = static_cast<const uint8_t*>(samples);
    // 2-bit: keep every packed 21-bit field below 2^21 by spilling into the
    // wide arrays first, and split runs too long for one pass.
    const int64_t L = p->g.L;
    const int64_t cap = (PCAL_F21_LIMIT - 2) * L / 16 * 16;
    while (n > 0) {
        int64_t take = n;
        if (p->g.format == PCAL_2BIT) {
            if (take > cap) take = cap;
            if ((p->since_spill + take) / L + 2 > PCAL_F21_LIMIT) {
                cudaError_t e = launch_spill2(p, s);
                if (e != cudaSuccess) return cuda_status(e);
                p->since_spill = 0;
                p->spilled = true;
            }
        }
        int rc = accumulate_run(p, d, take, s);
        if (rc != PCAL_OK) return rc;
        d += bytes_of(p, take);
        n -= take;
    }
    return PCAL_OK;
}

namespace {

int accumulate_host_impl(pcal_plan* p, const void* host, int64_t n, void* stream, bool wait) {
    if (!p || n < 0) return PCAL_EINVAL;
    if (n == 0) return PCAL_OK;
    if (!host) return PCAL_EINVAL;
    if (p->g.format == PCAL_2BIT && n % 4 != 0) return PCAL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!p->d_stage[0]) {
        e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaMalloc(&p->d_stage[i], kStageBytes);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->stage_ev[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->copied_ev[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_status(e);
        p->stage_bytes = kStageBytes;
    }
    // Chunks are whole bulk rows so that only the last one has a ragged tail.
    const int64_t row_bytes = bytes_of(p, p->g.row_samples);
    int64_t chunk = (int64_t)p->stage_bytes / row_bytes * row_bytes;
    if (chunk <= 0) chunk = (int64_t)p->stage_bytes / 16 * 16;
    const uint8_t* h = static_cast<const uint8_t*>(host);
    int64_t left = bytes_of(p, n);
    int j = 0;
    while (left > 0) {
        const int64_t b = left < chunk ? left : chunk;
        // Copies run on the plan's copy stream, folds on `s`: the copy of
        // chunk c+1 overlaps the fold of chunk c.  A staging buffer is
        // refilled only after the fold that read it has finished.
        e = cudaStreamWaitEvent(p->copy_stream, p->stage_ev[j], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_stage[j], h, (size_t)b, cudaMemcpyHostToDevice, p->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(p->copied_ev[j], p->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->copied_ev[j], 0);
        if (e != cudaSuccess) return cuda_status(e);
        int rc = pcal_accumulate(p, p->d_stage[j], samples_of(p, b), stream);
        if (rc != PCAL_OK) return rc;
        e = cudaEventRecord(p->stage_ev[j], s);
        if (e != cudaSuccess) return cuda_status(e);
        h += b;
        left -= b;
        j ^= 1;
    }
    // the host buffer may be reused once its copies are done
    if (wait) e = cudaStreamSynchronize(p->copy_stream);
    return cuda_status(e);
}

}  // namespace

extern "C" int pcal_accumulate_host(pcal_plan* p, const void* host, int64_t n, void* stream) {
    return accumulate_host_impl(p, host, n, stream, true);
}

extern "C" int pcal_accumulate_host_async(pcal_plan* p, const void* host, int64_t n, void* stream) {
    return accumulate_host_impl(p, host, n, stream, false);
}

extern "C" int pcal_finalize_device(pcal_plan* p, void* stream) {
    if (!p) return PCAL_EINVAL;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->last_stream;
    cudaError_t e = launch_finalize(p, s);
    if (e != cudaSuccess) return cuda_status(e);
    p->cur ^= 1;  // the next period adds into the other bin set
    p->last_stream = s;
    p->period_start = p->n_abs;
    p->since_spill = 0;
    p->spilled = false;
    p->results_valid = true;
    return PCAL_OK;
}

extern "C" int pcal_read_results(pcal_plan* p, double* phasors, double* amp, double* phase, double* unwrapped,
                                 double* td, double* sigma) {
    if (!p) return PCAL_EINVAL;
    if (!p->results_valid) return PCAL_EBUSY;
    const int64_t N = p->g.N;
    cudaError_t e = cudaMemcpyAsync(p->h_res, p->d_res, (5 * N + 3) * sizeof(double), cudaMemcpyDeviceToHost,
                                    p->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned int err = 0;
    e = cudaMemcpy(&err, p->d_err, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (err) return PCAL_ETIMEOUT;
    if (phasors) memcpy(phasors, p->h_res, 2 * N * sizeof(double));
    if (amp) memcpy(amp, p->h_res + 2 * N, N * sizeof(double));
    if (phase) memcpy(phase, p->h_res + 3 * N, N * sizeof(double));
    if (unwrapped) memcpy(unwrapped, p->h_res + 4 * N, N * sizeof(double));
    if (td) *td = p->h_res[5 * N];
    if (sigma) *sigma = p->h_res[5 * N + 1];
    return PCAL_OK;
}

extern "C" int pcal_finalize_async(pcal_plan* p, void* stream) {
    if (!p) return PCAL_EINVAL;
    const int64_t N = p->g.N;
    const size_t bytes = (5 * N + 3) * sizeof(double);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        if (!p->h_ring[i]) e = cudaMallocHost(reinterpret_cast<void**>(&p->h_ring[i]), bytes + sizeof(double));
        if (e == cudaSuccess && !p->ring_ev[i]) e = cudaEventCreateWithFlags(&p->ring_ev[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_status(e);
    const int rc = pcal_finalize_device(p, stream);
    if (rc != PCAL_OK) return rc;
    const int slot = (int)(p->ring_count % 2);
    double* h = p->h_ring[slot];
    e = cudaMemcpyAsync(h, p->d_res, bytes, cudaMemcpyDeviceToHost, p->last_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + 5 * N + 3, p->d_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, p->last_stream);
    if (e == cudaSuccess) e = cudaEventRecord(p->ring_ev[slot], p->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    ++p->ring_count;
    return PCAL_OK;
}

extern "C" int pcal_read_async_results(pcal_plan* p, int age, double* phasors, double* amp, double* phase,
                                       double* unwrapped, double* td, double* sigma) {
    if (!p || age < 0 || age > 1 || age >= p->ring_count) return PCAL_EINVAL;
    const int64_t N = p->g.N;
    const int slot = (int)((p->ring_count - 1 - age) % 2);
    const cudaError_t e = cudaEventSynchronize(p->ring_ev[slot]);
    if (e != cudaSuccess) return cuda_status(e);
    const double* h = p->h_ring[slot];
    unsigned int err;
    memcpy(&err, h + 5 * N + 3, sizeof(err));
    if (err) return PCAL_ETIMEOUT;
    if (phasors) memcpy(phasors, h, 2 * N * sizeof(double));
    if (amp) memcpy(amp, h + 2 * N, N * sizeof(double));
    if (phase) memcpy(phase, h + 3 * N, N * sizeof(double));
    if (unwrapped) memcpy(unwrapped, h + 4 * N, N * sizeof(double));
    if (td) *td = h[5 * N];
    if (sigma) *sigma = h[5 * N + 1];
    return PCAL_OK;
}

extern "C" int pcal_finalize(pcal_plan* p, double* phasors_out) {
    int rc = pcal_finalize_device(p, nullptr);
    if (rc != PCAL_OK) return rc;
    return pcal_read_results(p, phasors_out, nullptr, nullptr, nullptr, nullptr, nullptr);
}

extern "C" int pcal_read_post(pcal_plan* p, double* td_peak, double* peak_bin, double* bandpass_phase) {
    if (!p) return PCAL_EINVAL;
    if (!p->results_valid) return PCAL_EBUSY;
    const int64_t N = p->g.N;
    double* h = p->h_res + 5 * N + 3;
    cudaError_t e = cudaMemcpyAsync(h, p->d_res + 5 * N + 3, (N + 2) * sizeof(double), cudaMemcpyDeviceToHost,
                                    p->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (td_peak) *td_peak = h[0];
    if (peak_bin) *peak_bin = h[1];
    if (bandpass_phase) memcpy(bandpass_phase, h + 2, N * sizeof(double));
    return PCAL_OK;
}

extern "C" int pcal_get_delay(pcal_plan* p, double* td, double* sigma) {
    if (!p || !td || !sigma) return PCAL_EINVAL;
    if (!p->results_valid) return PCAL_EBUSY;
    const int64_t N = p->g.N;
    *td = p->h_res[5 * N];
    *sigma = p->h_res[5 * N + 1];
    return PCAL_OK;
}

extern "C" const double* pcal_result_device(const pcal_plan* p) { return p ? p->d_res : nullptr; }

extern "C" int pcal_get_bins(pcal_plan* p, void* host_out) {
    if (!p || !host_out) return PCAL_EINVAL;
    const int64_t L = p->g.L;
    cudaError_t e = flush_partials(p, p->last_stream);  // float32: pending fold partials into the bins
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (p->g.format == PCAL_I8) return cuda_status(cudaMemcpy(host_out, cur_acc8(p), L * 8, cudaMemcpyDeviceToHost));
    if (p->g.format == PCAL_F32) {
        // double-float bins -> FP64 on the host
        float* tmp = static_cast<float*>(malloc((size_t)L * 2 * sizeof(float)));
        if (!tmp) return PCAL_ENOMEM;
        e = cudaMemcpy(tmp, cur_accf(p), (size_t)L * 2 * sizeof(float), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (int64_t k = 0; k < L; ++k)
                static_cast<double*>(host_out)[k] = (double)tmp[2 * k] + (double)tmp[2 * k + 1];
        free(tmp);
        return cuda_status(e);
    }
    void* d_tmp = nullptr;
    e = cudaMalloc(&d_tmp, (size_t)L * 4 * 8);
    if (e == cudaSuccess) e = launch_export_bins(p, d_tmp, p->last_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d_tmp, (size_t)L * 4 * 8, cudaMemcpyDeviceToHost,
                                              p->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->last_stream);
    cudaFree(d_tmp);
    return cuda_status(e);
}

extern "C" int pcal_get_stats(const pcal_plan* p, pcal_stats* out) {
    if (!p || !out) return PCAL_EINVAL;
    *out = p->stats;
    out->n_abs = p->n_abs;
    out->n_period = p->n_abs - p->period_start;
    return PCAL_OK;
}
