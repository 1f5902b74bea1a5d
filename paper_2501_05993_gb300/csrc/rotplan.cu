// Long-period plans (pcal_rotplan_*): offsets whose combined period L is too
// long to fold (prime offsets; L above 2^20) or that are not whole hertz.
//
// There is no short period to fold over, so every sample is rotated by
// exp(-j*w_o*n) (Eq. 3) and added into bin n mod N (Eq. 2), as in the
// paper's own route, but in double-float: thread (lane, b) owns the samples
// n = b (mod N) with (n div N) = lane (mod lanes); its rotator advances by
// one double-float complex multiplication per sample and is re-seeded every
// kReseed samples from the exact phase frac(n * f_offset / fs), computed in
// double-double from f_offset/fs and taken through FP64 sincospi -- so the
// rotator error never accumulates over more than kReseed steps.  The sums
// are double-float; the finalize adds the lanes of each bin in double-float,
// runs the N-point DFT and the products of the folded path.
#include <math.h>
#include <string.h>

#include <new>

#include "df64.cuh"
#include "internal.cuh"

namespace {

using pcal_df::df;

constexpr int kReseed = 256;

struct RotAccArgs {
    const void* x;
    int64_t n, n0;
    int fmt;
    int N, lanes;
    double r_hi, r_lo;  // f_offset / fs as a double-double
    df lev[4];          // 2-bit code values
    float4* acc;        // [lanes][N]: re (hi, lo), im (hi, lo)
};

// frac(n * (r_hi + r_lo)) for 0 <= n < 2^52, about 1e-16 absolute: n is split
// into two exactly representable parts, each product into its rounded value
// and its exact error (fma), and only fractional parts are added.
__device__ __forceinline__ double frac_mul(int64_t n, double r_hi, double r_lo) {
    const double nh = (double)(n >> 26) * 67108864.0;
    const double nl = (double)(n & 0x3FFFFFF);
    const double p = nh * r_hi, e = fma(nh, r_hi, -p);
    const double q = nl * r_hi, g = fma(nl, r_hi, -q);
    double f = (p - floor(p)) + (q - floor(q));
    f += e + g + (double)n * r_lo;
    return f - floor(f);
}

// exp(-j*2*pi*c) as a double-float complex (re, im).
__device__ __forceinline__ void phasor_df(double c, df* re, df* im) {
    double s, co;
    sincospi(2.0 * c, &s, &co);
    s = -s;
    re->hi = (float)co;
    re->lo = (float)(co - (double)re->hi);
    im->hi = (float)s;
    im->lo = (float)(s - (double)im->hi);
}

__device__ __forceinline__ df sample_df(const RotAccArgs& a, int64_t i) {
    if (a.fmt == PCAL_I8) return df{(float)static_cast<const int8_t*>(a.x)[i], 0.f};
    if (a.fmt == PCAL_F32) return df{static_cast<const float*>(a.x)[i], 0.f};
    const int c = (static_cast<const uint8_t*>(a.x)[i >> 2] >> (2 * (int)(i & 3))) & 3;
    return a.lev[c];
}

__global__ void rotplan_acc_kernel(const __grid_constant__ RotAccArgs a) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)a.N * a.lanes) return;
    const int b = (int)(t % a.N), lane = (int)(t / a.N);
    const int64_t period = (int64_t)a.N * a.lanes;
    int64_t i = (((int64_t)lane * a.N + b - a.n0) % period + period) % period;
    if (i >= a.n) return;
    const float4 s0 = a.acc[t];
    df sr{s0.x, s0.y}, si{s0.z, s0.w};
    df step_re, step_im;
    phasor_df(frac_mul(period, a.r_hi, a.r_lo), &step_re, &step_im);
    df rr, ri;
    int k = 0;
    // Eight samples are loaded ahead of their rotations: one load per step on
    // the dependent chain left every step waiting for memory (163 Gsamples/s
    // on int8; 201 with the loads ahead; same sums, same order).
    constexpr int kAhead = 8;
    while (i < a.n) {
        df xs[kAhead];
#pragma unroll
        for (int u = 0; u < kAhead; ++u) xs[u] = i + u * period < a.n ? sample_df(a, i + u * period) : df{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < kAhead; ++u) {
            if (i >= a.n) break;
            if (k % kReseed == 0) phasor_df(frac_mul(a.n0 + i, a.r_hi, a.r_lo), &rr, &ri);
            const df x = xs[u];
            sr = pcal_df::add(sr, pcal_df::mul(x, rr));
            si = pcal_df::add(si, pcal_df::mul(x, ri));
            // next rotator: (rr + j ri) * (step_re + j step_im)
            const df nr = pcal_df::sub(pcal_df::mul(rr, step_re), pcal_df::mul(ri, step_im));
            const df ni = pcal_df::add(pcal_df::mul(rr, step_im), pcal_df::mul(ri, step_re));
            rr = nr;
            ri = ni;
            i += period;
            ++k;
        }
    }
    a.acc[t] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
}

__global__ void rotplan_twiddles_kernel(float2* twN, int N) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)N, &s, &c);
    twN[m] = make_float2((float)c, (float)-s);
}

}  // namespace

struct pcal_rotplan {
    int64_t fs, fc;
    double fo;
    int N, fmt, lanes;
    double r_hi, r_lo;
    double levels[4];
    int64_t n_abs, period_start;
    float4* d_acc;
    float2* d_twN;
    double* d_res;  // 5N+3 results, then N+2 post-processing values
    double* h_res;
    cudaStream_t last_stream;
    bool results_valid;
};

extern "C" int pcal_rotplan_create(double fs, double f_comb, double f_offset, int N, int sample_format,
                                   pcal_rotplan** out) {
    if (!out) return PCAL_EINVAL;
    *out = nullptr;
    if (!(fs > 0) || !(f_comb > 0) || fs != floor(fs) || f_comb != floor(f_comb) || fs > 9.0e15 ||
        !(f_offset >= 0.0) || !(f_offset < f_comb) || (sample_format != PCAL_F32 && sample_format != PCAL_I8 &&
                                                        sample_format != PCAL_2BIT))
        return PCAL_EINVAL;
    const int64_t ifs = (int64_t)fs, ifc = (int64_t)f_comb;
    if (ifs % ifc != 0 || N != ifs / ifc) return PCAL_EINVAL;
    if (N > PCAL_BATCH_MAX_N) return PCAL_ETOOLARGE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        (void)cudaGetLastError();
        return PCAL_ECUDA;
    }
    pcal_rotplan* r = new (std::nothrow) pcal_rotplan();
    if (!r) return PCAL_ENOMEM;
    r->fs = ifs;
    r->fc = ifc;
    r->fo = f_offset;
    r->N = N;
    r->fmt = sample_format;
    // about 1024 threads per SM, at least one lane
    r->lanes = (int)((int64_t)sms * 1024 / N);
    if (r->lanes < 1) r->lanes = 1;
    r->r_hi = f_offset / fs;
    r->r_lo = fma(-r->r_hi, fs, f_offset) / fs;
    const double lv[4] = {-3.3359, -1.0, 1.0, 3.3359};
    memcpy(r->levels, lv, sizeof(lv));
    r->n_abs = r->period_start = 0;
    r->last_stream = nullptr;
    r->results_valid = false;
    cudaError_t e = cudaMalloc(&r->d_acc, sizeof(float4) * (size_t)N * r->lanes);
    if (e == cudaSuccess) e = cudaMemset(r->d_acc, 0, sizeof(float4) * (size_t)N * r->lanes);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_twN, sizeof(float2) * N);
    if (e == cudaSuccess) e = cudaMalloc(&r->d_res, sizeof(double) * (6 * (size_t)N + 5));
    if (e == cudaSuccess) e = cudaMallocHost(&r->h_res, sizeof(double) * (6 * (size_t)N + 5));
    if (e == cudaSuccess) {
        rotplan_twiddles_kernel<<<(N + 255) / 256, 256>>>(r->d_twN, N);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        pcal_rotplan_destroy(r);
        return e == cudaErrorMemoryAllocation ? PCAL_ENOMEM : PCAL_ECUDA;
    }
    *out = r;
    return PCAL_OK;
}

extern "C" int pcal_rotplan_destroy(pcal_rotplan* r) {
    if (!r) return PCAL_OK;
    if (r->last_stream) cudaStreamSynchronize(r->last_stream);
    cudaFree(r->d_acc);
    cudaFree(r->d_twN);
    cudaFree(r->d_res);
    if (r->h_res) cudaFreeHost(r->h_res);
    (void)cudaGetLastError();
    delete r;
    return PCAL_OK;
}

extern "C" int pcal_rotplan_set_levels(pcal_rotplan* r, const double levels[4]) {
    if (!r || !levels) return PCAL_EINVAL;
    memcpy(r->levels, levels, sizeof(r->levels));
    return PCAL_OK;
}

extern "C" int pcal_rotplan_accumulate(pcal_rotplan* r, const void* samples, int64_t n, void* stream) {
    if (!r || n < 0 || (n > 0 && !samples)) return PCAL_EINVAL;
    if (r->fmt == PCAL_2BIT && n % 4 != 0) return PCAL_EINVAL;
    if (r->n_abs + n >= (1LL << 52)) return PCAL_ETOOLARGE;
    if (n == 0) return PCAL_OK;
    RotAccArgs a{};
    a.x = samples;
    a.n = n;
    a.n0 = r->n_abs;
    a.fmt = r->fmt;
    a.N = r->N;
    a.lanes = r->lanes;
    a.r_hi = r->r_hi;
    a.r_lo = r->r_lo;
    for (int c = 0; c < 4; ++c) {
        a.lev[c].hi = (float)r->levels[c];
        a.lev[c].lo = (float)(r->levels[c] - (double)a.lev[c].hi);
    }
    a.acc = r->d_acc;
    const int64_t threads = (int64_t)r->N * r->lanes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rotplan_acc_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return PCAL_ECUDA;
    r->n_abs += n;
    r->last_stream = s;
    return PCAL_OK;
}

extern "C" int pcal_rotplan_finalize_device(pcal_rotplan* r, void* stream) {
    if (!r) return PCAL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t M = r->n_abs - r->period_start;
    cudaError_t e = launch_rot_finalize(r->d_acc, r->lanes, r->N, (double)r->fs, (double)r->fc, M, r->d_twN, r->d_res,
                                        s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_acc, 0, sizeof(float4) * (size_t)r->N * r->lanes, s);
    if (e != cudaSuccess) return PCAL_ECUDA;
    r->period_start = r->n_abs;
    r->last_stream = s;
    r->results_valid = true;
    return PCAL_OK;
}

extern "C" int pcal_rotplan_read_results(pcal_rotplan* r, double* phasors, double* amp, double* phase,
                                         double* unwrapped, double* td, double* sigma, double* td_peak,
                                         double* bandpass_phase) {
    if (!r) return PCAL_EINVAL;
    if (!r->results_valid) return PCAL_EBUSY;
    const int64_t N = r->N;
    cudaError_t e = cudaMemcpyAsync(r->h_res, r->d_res, sizeof(double) * (6 * N + 5), cudaMemcpyDeviceToHost,
                                    r->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->last_stream);
    if (e != cudaSuccess) return PCAL_ECUDA;
    const double* h = r->h_res;
    if (phasors) memcpy(phasors, h, sizeof(double) * 2 * N);
    if (amp) memcpy(amp, h + 2 * N, sizeof(double) * N);
    if (phase) memcpy(phase, h + 3 * N, sizeof(double) * N);
    if (unwrapped) memcpy(unwrapped, h + 4 * N, sizeof(double) * N);
    if (td) *td = h[5 * N];
    if (sigma) *sigma = h[5 * N + 1];
    if (td_peak) *td_peak = h[5 * N + 3];
    if (bandpass_phase) memcpy(bandpass_phase, h + 5 * N + 5, sizeof(double) * N);
    return PCAL_OK;
}
