// Serving (pcal_server_*): continuous batching of many live streams.
//
// Streams open and close at any time.  A stream is admitted when its device
// memory -- bins, rotator table, results and a ring of recent samples -- fits
// in the server's HBM budget (one device allocation carved by a first-fit
// arena with coalescing free blocks); otherwise it waits in a queue and is
// admitted as soon as closed streams give memory back.
//
// Clients submit chunks of samples from host memory; each chunk is copied
// into its stream's device ring.  One scheduler thread repeatedly gathers
// every stream's pending samples (up to the end of the stream's current
// integration period), folds all of them with ONE persistent launch of the
// batched fold kernel, finalizes (one launch, a cluster per stream) the
// streams whose period just completed, and copies their results to pinned
// host memory.  Work submitted while a launch runs joins the next one: up to
// kSlots iterations are in flight on the compute stream, so copies, folds and
// finalizes of different streams overlap.  A host callback at the end of
// every iteration frees ring space, publishes the results with their
// latency (last sample of the period submitted -> results on the host) and
// returns the memory of closed streams.  A period's latency runs from the
// arrival of the chunk that brought its last sample -- the time the client
// stamps on it (pcal_server_submit_many_at), else the return of its submit --
// to the moment its results are on the host, so the ingest copy, any wait
// for ring space or admission and the client's own lag are inside it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "arena.h"
#include "internal.cuh"

namespace {

constexpr int kSlots = 4;  // iterations in flight

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

using pcal_arena::Arena;

enum StreamState { kQueued, kActive, kClosing, kReleased };

struct SrvStream {
    int id = -1;
    int slot = -1;
    StreamState state = kQueued;
    pcal_channel_desc desc{};
    pcal_geometry g{};
    int spb = 1;                 // samples per byte
    size_t off = 0, bytes = 0;   // arena block
    uint8_t* ring = nullptr;
    int64_t ring_bytes = 0;
    int64_t submitted = 0;       // samples in the ring (absolute count)
    int64_t launched = 0;        // samples handed to fold launches
    int64_t completed = 0;       // samples whose launches finished
    int64_t period_samples = 0;
    int64_t period_end = 0;      // end of the current period (absolute sample)
    int64_t period_index = 0;
    bool release_pending = false;
    std::deque<std::pair<int64_t, double>> arrivals;  // (end sample of a chunk, its arrival time)
    double* h_res = nullptr;     // pinned, 5N+3 doubles
};

struct Published {
    pcal_server_result r;
    std::vector<double> phasors;
};

struct IterInfo;

}  // namespace

// One piece of a submit's ingest: bytes from host memory the GPU can read
// into a stream's ring.
struct CopyPiece {
    const uint8_t* src;
    uint8_t* dst;
    long long bytes;
};

struct pcal_server {
    pcal_server_config cfg;
    int device = 0, num_sms = 0;
    uint8_t* d_mem = nullptr;
    Arena arena;
    std::deque<SrvStream> streams;    // by id (a deque: references stay valid as streams are added)
    std::vector<int> slot_owner;      // slot -> stream id or -1
    std::deque<int> queue;            // waiting for admission
    BatchChan* d_ch = nullptr;
    BatchChan* h_ch = nullptr;        // pinned mirror of the device records
    pcal_schedule sched{};
    int cw_max = 224;
    // launches
    cudaStream_t compute = nullptr, copy = nullptr;
    void* h_desc[kSlots] = {};
    void* d_desc[kSlots] = {};
    size_t desc_cap = 0;
    cudaEvent_t desc_ev[kSlots] = {};
    bool desc_used[kSlots] = {};
    int desc_next = 0;
    unsigned long long* d_ctr = nullptr;
    unsigned int* d_err = nullptr;
    // ingest: host chunks the GPU can read are gathered by one kernel per
    // submit (hundreds of small copies cost the copy engine more than the
    // link); the piece list lives in pinned, mapped memory
    int pageable_access = 0;          // the device reads pageable host memory
    CopyPiece* h_pieces = nullptr;
    CopyPiece* d_pieces = nullptr;
    int pieces_cap = 0;
    // threads
    std::mutex mu;
    std::mutex copy_mu;
    std::condition_variable cv_work, cv_space, cv_results, cv_idle;
    std::thread worker;
    bool stop = false;
    bool admit_dirty = false;
    int in_flight = 0;
    std::deque<Published> results;
    std::vector<double> latencies;
    pcal_server_stats stats{};
    int error = PCAL_OK;
};

namespace {

constexpr long long kPieceBytes = 256 << 10;  // gather work unit

// Block b copies pieces b, b + gridDim.x, ...: 16-byte words when the piece
// is 16-byte aligned at both ends and in length, bytes otherwise.  The host
// memory reads are issued four at a time per thread to keep the link busy.
__global__ void gather_kernel(const CopyPiece* __restrict__ pieces, int n) {
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        const CopyPiece p = pieces[b];
        const uintptr_t al = reinterpret_cast<uintptr_t>(p.src) | reinterpret_cast<uintptr_t>(p.dst) |
                             static_cast<uintptr_t>(p.bytes);
        if ((al & 15) == 0) {
            const uint4* src = reinterpret_cast<const uint4*>(p.src);
            uint4* dst = reinterpret_cast<uint4*>(p.dst);
            const long long n16 = p.bytes / 16, step = 4ll * blockDim.x;
            for (long long i = threadIdx.x; i < n16; i += step) {
                uint4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i + u * blockDim.x < n16) v[u] = src[i + u * blockDim.x];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i + u * blockDim.x < n16) dst[i + u * blockDim.x] = v[u];
            }
        } else {
            for (long long i = threadIdx.x; i < p.bytes; i += blockDim.x) p.dst[i] = p.src[i];
        }
    }
}

// Address through which the device reads host buffer `p`, or null when it
// cannot (pageable memory without pageable-memory access).
const uint8_t* device_view(const pcal_server* s, const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return s->pageable_access ? static_cast<const uint8_t*>(p) : nullptr;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer) return static_cast<const uint8_t*>(at.devicePointer);
    if (at.type == cudaMemoryTypeUnregistered && s->pageable_access) return static_cast<const uint8_t*>(p);
    return nullptr;
}

struct IterInfo {
    pcal_server* s;
    std::vector<std::pair<int, int64_t>> done;  // stream id, completed position
    struct Fin {
        int id;
        int64_t period, n, end;
    };
    std::vector<Fin> fins;
    std::vector<int> release;  // stream ids whose memory returns
};

// Host callback at the end of one iteration (no CUDA calls allowed here).
void CUDART_CB iteration_done(void* p) {
    IterInfo* it = static_cast<IterInfo*>(p);
    pcal_server* s = it->s;
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& d : it->done) {
            SrvStream& st = s->streams[d.first];
            if (d.second > st.completed) st.completed = d.second;
        }
        for (const IterInfo::Fin& f : it->fins) {
            SrvStream& st = s->streams[f.id];
            // arrival of the chunk that brought the period's last sample
            double t_arr = t;
            while (!st.arrivals.empty() && st.arrivals.front().first < f.end) st.arrivals.pop_front();
            if (!st.arrivals.empty()) t_arr = st.arrivals.front().second;
            const int64_t N = st.g.N;
            Published pub;
            pub.r.stream = f.id;
            pub.r.n_tones = (int32_t)N;
            pub.r.period = f.period;
            pub.r.n_samples = f.n;
            pub.r.td_s = st.h_res[5 * N];
            pub.r.sigma_td_s = st.h_res[5 * N + 1];
            pub.r.latency_s = t - t_arr;
            pub.r.td_peak_s = st.h_res[5 * N + 3];
            pub.phasors.assign(st.h_res, st.h_res + 2 * N);
            s->latencies.push_back(pub.r.latency_s);
            s->results.push_back(std::move(pub));
            s->stats.periods += 1;
        }
        for (int id : it->release) {
            SrvStream& st = s->streams[id];
            s->arena.release(st.off, st.bytes);
            s->slot_owner[st.slot] = -1;
            st.state = kReleased;
            st.slot = -1;
            s->stats.active -= 1;
            s->admit_dirty = true;
        }
        s->in_flight -= 1;
    }
    s->cv_space.notify_all();
    s->cv_results.notify_all();
    s->cv_idle.notify_all();
    s->cv_work.notify_all();
    delete it;
}

// Admit queued streams that fit (worker thread, lock held): arena block,
// slot, zeroed bins, rotator tables, device record.
void admit_queued(pcal_server* s) {
    s->admit_dirty = false;
    while (!s->queue.empty()) {
        SrvStream& st = s->streams[s->queue.front()];
        int slot = -1;
        for (int i = 0; i < (int)s->slot_owner.size(); ++i)
            if (s->slot_owner[i] < 0) {
                slot = i;
                break;
            }
        if (slot < 0) return;
        size_t off = 0;
        if (!s->arena.alloc(st.bytes, &off)) return;
        s->queue.pop_front();
        st.off = off;
        st.slot = slot;
        s->slot_owner[slot] = st.id;
        BatchChan& C = s->h_ch[slot];
        batch_fill_chan(C, st.g, st.desc.f_comb, s->sched);
        uint8_t* base = s->d_mem + off;
        batch_place_chan(C, st.g, base);
        const size_t chan_bytes = batch_chan_bytes(st.g);
        st.ring = base + chan_bytes;
        cudaError_t e = cudaMemsetAsync(base, 0, chan_bytes, s->compute);
        if (e == cudaSuccess) e = batch_launch_tables(C, st.g, s->compute);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_ch + slot, &C, sizeof(BatchChan), cudaMemcpyHostToDevice, s->compute);
        if (e != cudaSuccess) s->error = PCAL_ECUDA;
        st.state = kActive;
        s->stats.admitted += 1;
        s->stats.queued -= 1;
        s->stats.active += 1;
    }
}

bool has_work(pcal_server* s) {
    if (s->admit_dirty && !s->queue.empty()) return true;
    for (const SrvStream& st : s->streams) {
        if (st.state == kActive && st.submitted > st.launched) return true;
        if (st.state == kClosing && !st.release_pending) return true;
    }
    return false;
}

void worker_loop(pcal_server* s) {
    cudaSetDevice(s->device);
    BatchShape sh;
    batch_shape(s->sched, s->cw_max, s->num_sms, &sh);
    for (;;) {
        std::vector<BatchRegion> regions;
        std::vector<int> fin_slots;
        IterInfo* info = new IterInfo();
        info->s = s;
        int max_n = 1;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || has_work(s); });
            if (s->stop && !has_work(s)) {
                delete info;
                break;
            }
            if (s->admit_dirty) {
                admit_queued(s);
                s->cv_space.notify_all();  // submits waiting for admission
            }
            for (SrvStream& st : s->streams) {
                if (st.state != kActive && st.state != kClosing) continue;
                if (st.submitted > st.launched) {
                    const int64_t end = std::min(st.submitted, st.period_end);
                    const int64_t n = end - st.launched;
                    // ring coordinates in bytes; split where the ring wraps
                    int64_t b0 = (st.launched / st.spb) % st.ring_bytes;
                    int64_t nb = n / st.spb, off = 0;
                    while (nb > 0) {
                        const int64_t take = std::min(nb, st.ring_bytes - b0);
                        regions.push_back(BatchRegion{st.slot, st.ring + b0, take * st.spb, off});
                        off += take * st.spb;
                        nb -= take;
                        b0 = 0;
                    }
                    st.launched = end;
                    info->done.push_back({st.id, end});
                    if (end == st.period_end) {
                        fin_slots.push_back(st.slot);
                        info->fins.push_back({st.id, st.period_index, st.period_samples, end});
                        if (st.g.N > max_n) max_n = (int)st.g.N;
                        st.period_index += 1;
                        st.period_end += st.period_samples;
                    }
                }
                if (st.state == kClosing && !st.release_pending && st.launched == st.submitted) {
                    st.release_pending = true;
                    info->release.push_back(st.id);
                }
            }
            s->in_flight += 1;
        }
        // descriptors of this iteration
        BatchCallDesc d;
        int rc = batch_build(s->h_ch, (int)s->slot_owner.size(), regions, sh, fin_slots, &d);
        cudaError_t e = rc == PCAL_OK ? cudaSuccess : cudaErrorInvalidValue;
        const int i = s->desc_next;
        s->desc_next = (i + 1) % kSlots;
        if (e == cudaSuccess && s->desc_used[i]) e = cudaEventSynchronize(s->desc_ev[i]);
        if (e == cudaSuccess && d.blob.size() > s->desc_cap) {
            for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
                if (s->desc_used[k]) e = cudaEventSynchronize(s->desc_ev[k]);
                if (s->h_desc[k]) cudaFreeHost(s->h_desc[k]);
                if (s->d_desc[k]) cudaFree(s->d_desc[k]);
                s->h_desc[k] = s->d_desc[k] = nullptr;
                s->desc_used[k] = false;
            }
            const size_t cap = align_up(d.blob.size() * 2, 4096);
            for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
                e = cudaMallocHost(&s->h_desc[k], cap);
                if (e == cudaSuccess) e = cudaMalloc(&s->d_desc[k], cap);
            }
            if (e == cudaSuccess) s->desc_cap = cap;
        }
        int launches = 0;
        if (e == cudaSuccess) {
            memcpy(s->h_desc[i], d.blob.data(), d.blob.size());
            e = cudaMemcpyAsync(s->d_desc[i], s->h_desc[i], d.blob.size(), cudaMemcpyHostToDevice, s->compute);
        }
        if (e == cudaSuccess && !regions.empty())
            e = batch_launch_fold(d, s->d_desc[i], s->d_ch, (int)s->slot_owner.size(), s->d_ctr, sh, s->d_err,
                                  s->compute, &launches);
        if (e == cudaSuccess && !fin_slots.empty()) {
            const int* d_list = reinterpret_cast<const int*>(static_cast<uint8_t*>(s->d_desc[i]) + d.off_list);
            e = launch_batch_finalize(s->d_ch, (int)fin_slots.size(), max_n, d_list, s->compute);
            launches += 1;
            for (const IterInfo::Fin& f : info->fins) {
                if (e != cudaSuccess) break;
                const SrvStream& st = s->streams[f.id];
                e = cudaMemcpyAsync(st.h_res, s->h_ch[st.slot].res, sizeof(double) * (6 * st.g.N + 5),
                                    cudaMemcpyDeviceToHost, s->compute);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(s->desc_ev[i], s->compute);
        if (e == cudaSuccess) s->desc_used[i] = true;
        if (e == cudaSuccess) e = cudaLaunchHostFunc(s->compute, iteration_done, info);
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.launches += launches;
        if (e != cudaSuccess) {
            s->error = PCAL_ECUDA;
            s->in_flight -= 1;
            delete info;
            s->cv_idle.notify_all();
            s->cv_space.notify_all();
        }
    }
}

}  // namespace

extern "C" int pcal_server_create(const pcal_server_config* cfg, pcal_server** out) {
    if (!out) return PCAL_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->hbm_budget_bytes <= 0 || cfg->max_streams <= 0 || cfg->max_streams > PCAL_MAX_BATCH ||
        !(cfg->period_s > 0.0) || !(cfg->ring_s > 0.0))
        return PCAL_EINVAL;
    pcal_server* s = new (std::nothrow) pcal_server();
    if (!s) return PCAL_ENOMEM;
    s->cfg = *cfg;
    s->sched = pcal_schedule{0, 32, 0, 90, 4, 224, {}};
    s->slot_owner.assign(cfg->max_streams, -1);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_mem, (size_t)cfg->hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ch, sizeof(BatchChan) * cfg->max_streams);
    if (e == cudaSuccess) e = cudaMemset(s->d_ch, 0, sizeof(BatchChan) * cfg->max_streams);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_ch, sizeof(BatchChan) * cfg->max_streams);
    if (e == cudaSuccess) memset(static_cast<void*>(s->h_ch), 0, sizeof(BatchChan) * cfg->max_streams);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctr, 256);
    if (e == cudaSuccess) e = cudaMemset(s->d_ctr, 0, 256);  // each fold leaves its counters zero
    if (e == cudaSuccess) e = cudaMalloc(&s->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(s->d_err, 0, 256);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess &&
        cudaDeviceGetAttribute(&s->pageable_access, cudaDevAttrPageableMemoryAccess, s->device) != cudaSuccess) {
        (void)cudaGetLastError();
        s->pageable_access = 0;
    }
    for (int k = 0; k < kSlots && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&s->desc_ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = batch_prepare_fold();
    if (e == cudaSuccess) e = prepare_batch_finalize();
    // First use must not stall a live stream: load the gather kernel now (modules load lazily, on first
    // launch) and size the pinned piece list and the descriptor buffers for every stream at once.
    if (e == cudaSuccess) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, gather_kernel);
    }
    if (e == cudaSuccess) {
        const int cap = 16 * cfg->max_streams;
        e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_pieces), sizeof(CopyPiece) * cap, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_pieces), s->h_pieces, 0);
        if (e == cudaSuccess) s->pieces_cap = cap;
    }
    if (e == cudaSuccess) {
        const size_t cap = align_up((size_t)cfg->max_streams * 8192 + 65536, 4096);
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
            e = cudaMallocHost(&s->h_desc[k], cap);
            if (e == cudaSuccess) e = cudaMalloc(&s->d_desc[k], cap);
        }
        if (e == cudaSuccess) s->desc_cap = cap;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        const bool oom = e == cudaErrorMemoryAllocation;
        pcal_server_destroy(s);
        return oom ? PCAL_ENOMEM : PCAL_ECUDA;
    }
    s->arena.reset((size_t)cfg->hbm_budget_bytes);
    s->stats.hbm_budget = cfg->hbm_budget_bytes;
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return PCAL_OK;
}

extern "C" int pcal_server_destroy(pcal_server* s) {
    if (!s) return PCAL_OK;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    if (s->compute) cudaStreamSynchronize(s->compute);
    for (SrvStream& st : s->streams)
        if (st.h_res) cudaFreeHost(st.h_res);
    for (int k = 0; k < kSlots; ++k) {
        if (s->h_desc[k]) cudaFreeHost(s->h_desc[k]);
        if (s->d_desc[k]) cudaFree(s->d_desc[k]);
        if (s->desc_ev[k]) cudaEventDestroy(s->desc_ev[k]);
    }
    if (s->copy) cudaStreamSynchronize(s->copy);
    if (s->h_pieces) cudaFreeHost(s->h_pieces);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    cudaFree(s->d_mem);
    cudaFree(s->d_ch);
    if (s->h_ch) cudaFreeHost(s->h_ch);
    cudaFree(s->d_ctr);
    cudaFree(s->d_err);
    (void)cudaGetLastError();
    delete s;
    return PCAL_OK;
}

namespace {

// Geometry, period and device footprint of a stream for a server config.
int stream_layout(const pcal_server_config& cfg, const pcal_channel_desc& desc, SrvStream* st) {
    if (desc.sample_format != PCAL_2BIT && desc.sample_format != PCAL_I8) return PCAL_EINVAL;
    int rc = pcal_plan_geometry(desc.fs, desc.f_comb, desc.f_offset, desc.N, desc.sample_format, &st->g);
    if (rc != PCAL_OK) return rc;
    if (st->g.N > PCAL_BATCH_MAX_N) return PCAL_ETOOLARGE;
    st->desc = desc;
    st->spb = desc.sample_format == PCAL_2BIT ? 4 : 1;
    const double per = desc.fs * cfg.period_s;
    st->period_samples = (int64_t)llround(per);
    if (fabs(per - (double)st->period_samples) > 1e-6 || st->period_samples <= 0 || st->period_samples % 4 != 0)
        return PCAL_EINVAL;
    st->period_end = st->period_samples;
    st->ring_bytes = (int64_t)align_up((size_t)ceil(desc.fs * cfg.ring_s / st->spb), 256);
    st->bytes = batch_chan_bytes(st->g) + (size_t)st->ring_bytes;
    return PCAL_OK;
}

}  // namespace

extern "C" int pcal_server_stream_bytes(const pcal_server_config* cfg, const pcal_channel_desc* desc, int64_t* out) {
    if (!cfg || !desc || !out || !(cfg->period_s > 0.0) || !(cfg->ring_s > 0.0)) return PCAL_EINVAL;
    SrvStream st;
    const int rc = stream_layout(*cfg, *desc, &st);
    if (rc == PCAL_OK) *out = (int64_t)align_up(st.bytes, 256);
    return rc;
}

extern "C" int pcal_server_open(pcal_server* s, const pcal_channel_desc* desc, int* stream_id) {
    if (!s || !desc || !stream_id) return PCAL_EINVAL;
    SrvStream st;
    const int rc = stream_layout(s->cfg, *desc, &st);
    if (rc != PCAL_OK) return rc;
    if (align_up(st.bytes, 256) > (size_t)s->cfg.hbm_budget_bytes) return PCAL_ENOMEM;
    if (cudaMallocHost(&st.h_res, sizeof(double) * (6 * st.g.N + 5)) != cudaSuccess) return PCAL_ENOMEM;
    std::lock_guard<std::mutex> lk(s->mu);
    st.id = (int)s->streams.size();
    s->streams.push_back(st);
    s->queue.push_back(st.id);
    s->stats.queued += 1;
    s->admit_dirty = true;
    *stream_id = st.id;
    s->cv_work.notify_all();
    return PCAL_OK;
}

extern "C" double pcal_clock_s(void) { return now_s(); }

extern "C" int pcal_server_submit_many_at(pcal_server* s, int count, const int* ids, const void* const* host,
                                          const int64_t* n, const double* arrival_s) {
    if (!s || count < 0 || (count > 0 && (!ids || !host || !n))) return PCAL_EINVAL;
    for (int k = 0; arrival_s && k < count; ++k)
        if (!(arrival_s[k] == arrival_s[k])) return PCAL_EINVAL;  // NaN
    std::vector<int64_t> pos(count);
    {
        std::unique_lock<std::mutex> lk(s->mu);
        for (int k = 0; k < count; ++k) {
            if (ids[k] < 0 || ids[k] >= (int)s->streams.size() || n[k] < 0) return PCAL_EINVAL;
            SrvStream& st = s->streams[ids[k]];
            if (st.state == kClosing || st.state == kReleased) return PCAL_EINVAL;
            if (n[k] % st.spb != 0 || n[k] > st.ring_bytes * st.spb) return PCAL_EINVAL;
            for (int j = 0; j < k; ++j)
                if (ids[j] == ids[k]) return PCAL_EINVAL;  // one chunk per stream per call
            // wait for admission and for ring space
            s->cv_space.wait(lk, [&] {
                return s->error != PCAL_OK ||
                       (st.state == kActive && st.submitted + n[k] - st.completed <= st.ring_bytes * st.spb);
            });
            if (s->error != PCAL_OK) return s->error;
            pos[k] = st.submitted;
        }
    }
    // copy into the rings (split where a ring wraps), then wait for the copies:
    // chunks the device can read go to one gather launch, the others to the
    // copy engine
    int64_t bytes = 0;
    {
        std::lock_guard<std::mutex> cl(s->copy_mu);
        cudaError_t e = cudaSuccess;
        std::vector<CopyPiece> pieces;
        for (int k = 0; k < count && e == cudaSuccess; ++k) {
            SrvStream& st = s->streams[ids[k]];
            const uint8_t* src = static_cast<const uint8_t*>(host[k]);
            const uint8_t* view = n[k] > 0 ? device_view(s, src) : nullptr;
            int64_t nb = n[k] / st.spb, b0 = (pos[k] / st.spb) % st.ring_bytes;
            bytes += nb;
            while (nb > 0 && e == cudaSuccess) {
                const int64_t take = std::min(nb, st.ring_bytes - b0);
                if (view) {
                    for (int64_t o = 0; o < take; o += kPieceBytes)
                        pieces.push_back(CopyPiece{view + o, st.ring + b0 + o, std::min<int64_t>(kPieceBytes, take - o)});
                    view += take;
                } else {
                    e = cudaMemcpyAsync(st.ring + b0, src, take, cudaMemcpyHostToDevice, s->copy);
                }
                src += take;
                nb -= take;
                b0 = 0;
            }
        }
        if (e == cudaSuccess && !pieces.empty()) {
            if ((int)pieces.size() > s->pieces_cap) {
                if (s->h_pieces) cudaFreeHost(s->h_pieces);
                s->h_pieces = nullptr;
                s->pieces_cap = 0;
                const int cap = (int)pieces.size() * 2;
                e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_pieces), sizeof(CopyPiece) * cap, cudaHostAllocMapped);
                if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_pieces), s->h_pieces, 0);
                if (e == cudaSuccess) s->pieces_cap = cap;
            }
            if (e == cudaSuccess) {
                memcpy(s->h_pieces, pieces.data(), sizeof(CopyPiece) * pieces.size());
                const int grid = std::min<int>((int)pieces.size(), 4 * s->num_sms);
                gather_kernel<<<grid, 256, 0, s->copy>>>(s->d_pieces, (int)pieces.size());
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy);
        if (e != cudaSuccess) return PCAL_ECUDA;
    }
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int k = 0; k < count; ++k) {
            SrvStream& st = s->streams[ids[k]];
            st.submitted += n[k];
            st.arrivals.push_back({st.submitted, arrival_s ? arrival_s[k] : t});
            s->stats.samples += n[k];
        }
        s->stats.bytes_h2d += bytes;
    }
    s->cv_work.notify_all();
    return PCAL_OK;
}

extern "C" int pcal_server_submit_many(pcal_server* s, int count, const int* ids, const void* const* host,
                                       const int64_t* n) {
    return pcal_server_submit_many_at(s, count, ids, host, n, nullptr);
}

extern "C" int pcal_server_submit(pcal_server* s, int stream_id, const void* host_samples, int64_t n) {
    return pcal_server_submit_many_at(s, 1, &stream_id, &host_samples, &n, nullptr);
}

extern "C" int pcal_server_close(pcal_server* s, int stream_id) {
    if (!s) return PCAL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (stream_id < 0 || stream_id >= (int)s->streams.size()) return PCAL_EINVAL;
    SrvStream& st = s->streams[stream_id];
    if (st.state == kQueued) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), stream_id));
        st.state = kReleased;
        s->stats.queued -= 1;
        return PCAL_OK;
    }
    if (st.state != kActive) return PCAL_EINVAL;
    st.state = kClosing;
    s->cv_work.notify_all();
    return PCAL_OK;
}

extern "C" int pcal_server_poll(pcal_server* s, pcal_server_result* out, double* phasors, int max_tones,
                                double timeout_s) {
    if (!s || !out) return PCAL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->results.empty() && timeout_s > 0)
        s->cv_results.wait_for(lk, std::chrono::duration<double>(timeout_s),
                               [&] { return !s->results.empty() || s->error != PCAL_OK; });
    if (s->results.empty()) return s->error != PCAL_OK ? s->error : 0;
    Published p = std::move(s->results.front());
    s->results.pop_front();
    lk.unlock();
    *out = p.r;
    if (phasors) {
        if (max_tones < p.r.n_tones) return PCAL_EINVAL;
        memcpy(phasors, p.phasors.data(), sizeof(double) * p.phasors.size());
    }
    return 1;
}

extern "C" int pcal_server_drain(pcal_server* s, double timeout_s) {
    if (!s) return PCAL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] {
        if (s->error != PCAL_OK) return true;
        if (s->in_flight > 0) return false;
        for (const SrvStream& st : s->streams)
            if ((st.state == kActive || st.state == kClosing) && st.launched < st.submitted) return false;
        for (const SrvStream& st : s->streams)
            if (st.state == kClosing) return false;
        return true;
    };
    if (!s->cv_idle.wait_for(lk, std::chrono::duration<double>(timeout_s), idle)) return PCAL_ETIMEOUT;
    return s->error;
}

extern "C" int pcal_server_get_stats(pcal_server* s, pcal_server_stats* out) {
    if (!s || !out) return PCAL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->hbm_in_use = (int64_t)s->arena.used();
    std::vector<double> v = s->latencies;
    out->p50_latency_s = out->p99_latency_s = out->max_latency_s = 0.0;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        out->p50_latency_s = v[(v.size() - 1) / 2];
        out->p99_latency_s = v[(size_t)((v.size() - 1) * 0.99)];
        out->max_latency_s = v.back();
    }
    unsigned int err = 0;
    if (cudaMemcpy(&err, s->d_err, sizeof(err), cudaMemcpyDeviceToHost) == cudaSuccess && err) return PCAL_ETIMEOUT;
    return s->error;
}
