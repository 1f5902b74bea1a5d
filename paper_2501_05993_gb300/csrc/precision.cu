// Precision study: the paper's own route in FP32, for comparison with the
// fold-first integer path (pcal_rotfold_*).
//
// Every sample is rotated by exp(-j*w_o*n) (Eq. 3) and added into bin
// n mod N (Eq. 2), then the bins are DFT'd -- with the rotator taken from an
// FP32 table of N_rot = fs/gcd(fs, f_offset) entries (Eq. 4; the precomputed
// vector of Sec. 2) or generated by the direct-form second-order resonator
// y[k+1] = 2 cos(d) y[k] - y[k-1] (Eq. 9, Sec. 2), and the products summed in
// FP32 either plainly or with Kahan compensation.  Each thread owns one bin
// b and one lane: samples n = b (mod N) whose index n div N is its lane
// (mod lanes), in sample order, so the order of every FP32 operation is
// fixed and a host emulation can reproduce it bit for bit.  The FP32
// accumulators live on the device across calls; the finalize adds the lanes
// of each bin in FP64 and runs the N-point DFT in FP64.
//
// The resonator here steps over one thread's samples, N*lanes apart, so its
// increment is d = 2*pi*f_offset*N*lanes/fs (mod 2*pi); it is seeded from
// the exact FP64 phase at each thread's first sample of every call.  (Stepped
// sample by sample, as in the paper, 2 cos(d) rounds to exactly 2 in FP32 for
// f_offset/fs below about 1e-4 and the recurrence degenerates -- the
// low-frequency distortion Sec. 2 warns about.)
#include <math.h>
#include <string.h>

#include <new>

#include "internal.cuh"

namespace {

struct RotFoldArgs {
    const void* x;
    int64_t n;        // samples of this call
    int64_t n0;       // absolute index of x[0]
    int fmt;          // PCAL_I8 or PCAL_F32
    int variant;      // PCAL_ROT_*
    int N;
    int lanes;
    int64_t n_rot;    // rotator period
    int64_t r_step;   // rotator index step per sample: f_offset/gcd(fs, f_offset) (mod n_rot)
    int64_t fs, fo;   // integral Hz
    const float2* table;  // exp(-j 2 pi m / n_rot), FP32
    float4* acc;      // per (lane, bin): sum re, sum im, compensation re, compensation im
};

__device__ __forceinline__ float sample_at(const RotFoldArgs& a, int64_t i) {
    if (a.fmt == PCAL_I8) return (float)static_cast<const int8_t*>(a.x)[i];
    return static_cast<const float*>(a.x)[i];
}

// exp(-j 2 pi (f * m mod fs) / fs) in FP64 (exact integer phase reduction).
__device__ __forceinline__ double2 phasor_fp64(int64_t f, int64_t m, int64_t fs) {
    const unsigned long long r = (unsigned long long)(((__int128)f * (__int128)m) % (__int128)fs);
    double s, c;
    sincospi(2.0 * (double)r / (double)fs, &s, &c);
    return make_double2(c, -s);
}

constexpr int kAhead = 8;  // samples (and table entries) loaded ahead of their use

__global__ void rotfold_kernel(RotFoldArgs a) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)a.N * a.lanes) return;
    const int b = (int)(t % a.N), lane = (int)(t / a.N);
    float4 s = a.acc[t];
    // first sample of this thread in the call: n0 + i == b (mod N), (n0 + i) div N == lane (mod lanes)
    const int64_t period = (int64_t)a.N * a.lanes;
    const int64_t want = (int64_t)lane * a.N + b;            // position within one period of N*lanes
    int64_t i = ((want - a.n0) % period + period) % period;
    if (i < a.n) {
        if (a.variant == PCAL_ROT_DFR) {
            const double2 p0 = phasor_fp64(a.fo, a.n0 + i, a.fs);
            const double2 p1 = phasor_fp64(a.fo, a.n0 + i + period, a.fs);
            const double2 pd = phasor_fp64(a.fo, period, a.fs);
            const float coef = (float)(2.0 * pd.x);
            float2 y0 = make_float2((float)p0.x, (float)p0.y), y1 = make_float2((float)p1.x, (float)p1.y);
            // samples loaded kAhead steps ahead of their use (same order of
            // operations; a load per step on the dependent chain waited for
            // memory every step)
            while (i < a.n) {
                float xs[kAhead];
#pragma unroll
                for (int u = 0; u < kAhead; ++u) xs[u] = i + u * period < a.n ? sample_at(a, i + u * period) : 0.f;
#pragma unroll
                for (int u = 0; u < kAhead; ++u) {
                    if (i >= a.n) break;
                    const float x = xs[u];
                    s.x = __fadd_rn(s.x, __fmul_rn(x, y0.x));
                    s.y = __fadd_rn(s.y, __fmul_rn(x, y0.y));
                    const float2 y2 = make_float2(__fsub_rn(__fmul_rn(coef, y1.x), y0.x),
                                                  __fsub_rn(__fmul_rn(coef, y1.y), y0.y));
                    y0 = y1;
                    y1 = y2;
                    i += period;
                }
            }
        } else {
            int64_t idx = (int64_t)(((__int128)(a.n0 + i) * a.r_step) % a.n_rot);
            const int64_t istep = (int64_t)(((__int128)period * a.r_step) % a.n_rot);
            const bool kahan = a.variant == PCAL_ROT_TABLE_KAHAN;
            while (i < a.n) {
                float xs[kAhead];
                float2 cs[kAhead];
                int64_t id = idx;
#pragma unroll
                for (int u = 0; u < kAhead; ++u) {
                    const bool in = i + u * period < a.n;
                    xs[u] = in ? sample_at(a, i + u * period) : 0.f;
                    cs[u] = in ? a.table[id] : make_float2(0.f, 0.f);
                    id += istep;
                    if (id >= a.n_rot) id -= a.n_rot;
                }
#pragma unroll
                for (int u = 0; u < kAhead; ++u) {
                    if (i >= a.n) break;
                    const float x = xs[u];
                    const float2 c = cs[u];
                    const float pr = __fmul_rn(x, c.x), pi = __fmul_rn(x, c.y);
                    if (kahan) {
                        const float yr = __fsub_rn(pr, s.z), yi = __fsub_rn(pi, s.w);
                        const float tr = __fadd_rn(s.x, yr), ti = __fadd_rn(s.y, yi);
                        s.z = __fsub_rn(__fsub_rn(tr, s.x), yr);
                        s.w = __fsub_rn(__fsub_rn(ti, s.y), yi);
                        s.x = tr;
                        s.y = ti;
                    } else {
                        s.x = __fadd_rn(s.x, pr);
                        s.y = __fadd_rn(s.y, pi);
                    }
                    idx += istep;
                    if (idx >= a.n_rot) idx -= a.n_rot;
                    i += period;
                }
            }
        }
    }
    a.acc[t] = s;
}

__global__ void rotfold_table_kernel(float2* table, int64_t n_rot) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n_rot; m += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)n_rot, &s, &c);
        table[m] = make_float2((float)c, (float)-s);
    }
}

// P[b] = sum over lanes of (sum - compensation), FP64, lane order.
__global__ void rotfold_combine_kernel(const float4* acc, int N, int lanes, double2* P) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= N) return;
    double re = 0.0, im = 0.0;
    for (int l = 0; l < lanes; ++l) {
        const float4 v = acc[(int64_t)l * N + b];
        re += (double)v.x - (double)v.z;
        im += (double)v.y - (double)v.w;
    }
    P[b] = make_double2(re, im);
}

// T_i = sum_b P[b] exp(-j 2 pi i b / N), FP64, one thread per tone.
__global__ void rotfold_dft_kernel(const double2* P, int N, double2* T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < N; ++b) {
        double sn, cs;
        sincospi(2.0 * (double)(((int64_t)i * b) % N) / (double)N, &sn, &cs);
        const double2 w = make_double2(cs, -sn);
        const double2 p = P[b];
        re += p.x * w.x - p.y * w.y;
        im += p.x * w.y + p.y * w.x;
    }
    T[i] = make_double2(re, im);
}

int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace

struct pcal_rotfold {
    int64_t fs, fc, fo;
    int N, fmt, variant, lanes;
    int64_t n_rot, r_step;
    int64_t n_abs;
    float2* d_table;
    float4* d_acc;
    double2* d_P;
    double2* d_T;
};

extern "C" int pcal_rotfold_create(double fs, double f_comb, double f_offset, int N, int sample_format, int variant,
                                   int lanes, pcal_rotfold** out) {
    if (!out) return PCAL_EINVAL;
    *out = nullptr;
    pcal_geometry g;
    int rc = pcal_plan_geometry(fs, f_comb, f_offset, N, sample_format, &g);
    if (rc != PCAL_OK) return rc;
    if ((sample_format != PCAL_I8 && sample_format != PCAL_F32) || variant < PCAL_ROT_TABLE ||
        variant > PCAL_ROT_DFR || lanes < 1 || lanes > 4096)
        return PCAL_EINVAL;
    pcal_rotfold* r = new (std::nothrow) pcal_rotfold();
    if (!r) return PCAL_ENOMEM;
    r->fs = g.fs;
    r->fc = g.f_comb;
    r->fo = g.f_offset;
    r->N = (int)g.N;
    r->fmt = sample_format;
    r->variant = variant;
    r->lanes = lanes;
    r->n_rot = g.N_rot;
    r->r_step = g.f_offset / gcd64(g.fs, g.f_offset == 0 ? g.fs : g.f_offset) % g.N_rot;
    r->n_abs = 0;
    cudaError_t e = cudaMalloc(&r->d_table, sizeof(float2) * r->n_rot);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_acc, sizeof(float4) * (size_t)r->N * lanes);
    if (e == cudaSuccess) e = cudaMemset(r->d_acc, 0, sizeof(float4) * (size_t)r->N * lanes);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_P, sizeof(double2) * r->N);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_T, sizeof(double2) * r->N);
    if (e == cudaSuccess) {
        int grid = (int)((r->n_rot + 255) / 256);
        if (grid > 1024) grid = 1024;
        rotfold_table_kernel<<<grid, 256>>>(r->d_table, r->n_rot);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        pcal_rotfold_destroy(r);
        return e == cudaErrorMemoryAllocation ? PCAL_ENOMEM : PCAL_ECUDA;
    }
    *out = r;
    return PCAL_OK;
}

extern "C" int pcal_rotfold_destroy(pcal_rotfold* r) {
    if (!r) return PCAL_OK;
    cudaFree(r->d_table);
    cudaFree(r->d_acc);
    cudaFree(r->d_P);
    cudaFree(r->d_T);
    (void)cudaGetLastError();
    delete r;
    return PCAL_OK;
}

extern "C" int pcal_rotfold_accumulate(pcal_rotfold* r, const void* samples, int64_t n, void* stream) {
    if (!r || n < 0 || (n > 0 && !samples)) return PCAL_EINVAL;
    if (n == 0) return PCAL_OK;
    RotFoldArgs a{};
    a.x = samples;
    a.n = n;
    a.n0 = r->n_abs;
    a.fmt = r->fmt;
    a.variant = r->variant;
    a.N = r->N;
    a.lanes = r->lanes;
    a.n_rot = r->n_rot;
    a.r_step = r->r_step;
    a.fs = r->fs;
    a.fo = r->fo;
    a.table = r->d_table;
    a.acc = r->d_acc;
    const int64_t threads = (int64_t)r->N * r->lanes;
    rotfold_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    if (cudaGetLastError() != cudaSuccess) return PCAL_ECUDA;
    r->n_abs += n;
    return PCAL_OK;
}

extern "C" int pcal_rotfold_finalize(pcal_rotfold* r, double* phasors_out, void* stream) {
    if (!r || !phasors_out) return PCAL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rotfold_combine_kernel<<<(r->N + 255) / 256, 256, 0, s>>>(r->d_acc, r->N, r->lanes, r->d_P);
    rotfold_dft_kernel<<<(r->N + 127) / 128, 128, 0, s>>>(r->d_P, r->N, r->d_T);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(phasors_out, r->d_T, sizeof(double2) * r->N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_acc, 0, sizeof(float4) * (size_t)r->N * r->lanes, s);
    return e == cudaSuccess ? PCAL_OK : PCAL_ECUDA;
}

extern "C" int pcal_rotfold_get_acc(pcal_rotfold* r, float* host_out) {
    if (!r || !host_out) return PCAL_EINVAL;
    return cudaMemcpy(host_out, r->d_acc, sizeof(float4) * (size_t)r->N * r->lanes, cudaMemcpyDeviceToHost) ==
                   cudaSuccess
               ? PCAL_OK
               : PCAL_ECUDA;
}
