// Finalize kernels of libpcal: from the L accumulated bins to N tone phasors
// and the delay (paper Sec. 2).
//
//   decode   S[k] from the exact bins (2-bit: the level table applied to the
//            per-code counts; int8/float32: the sums), FP64
//   rotate   R[k] = S[k] * exp(-j*2*pi*f_offset*k/fs)               (Eq. 3)
//   fold     P[b] = sum_m R[b + m*N]                                   (Eq. 2)
//   DFT      T_i = sum_b P[b] exp(-j*2*pi*i*b/N)          (DFT(P), Sec. 2)
//   products amp_i = 2|T_i|/M, phase arg(T_i)+pi/2 (sin model of Eq. 1),
//            unwrapped along the comb, delay = |T|^2-weighted LS slope of
//            phase versus f_i = i*f_comb + f_offset, divided by 2*pi
//            (phi_i = 2*pi*f_i*t_d, Eq. 1).
//
// The rotator phase is reduced exactly in integers, (f_offset/g * k) mod L,
// and looked up in the plan's FP64 table exp(-j*2*pi*m/L) (the paper's
// precomputed-rotator idea, Sec. 2 after Eq. 4, evaluated once per plan).
// Precision: decode, rotation and the fold to N run in FP64 (2 FMAs per
// bin); the N-point DFT runs in FP32 (N^2 complex MACs, spread over CTAs);
// the products and the least-squares fit use FP64 sums.
//
// Work split: the fold kernel gives each CTA whole residues b (so no two CTAs
// add into the same P[b]); the last CTA to finish (an atomic ticket, no
// waiting) runs the DFT for small N and the products.  For large N a second
// kernel spreads the DFT over CTAs and its last CTA runs the products.
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int kDftInFoldMaxN = 256;
constexpr int kDftTonesPerCta = 32;

struct FinArgs {
    int fmt;
    int bc;          // residues b per fold CTA
    int tpb;         // threads per residue (power of two)
    int64_t L, N, so;
    int64_t q, rem, a0;  // samples in bin k: q + ((k - a0) mod L < rem)
    double lev0, c_l, c_h, c_hl;
    double M, fc, fo;
    unsigned long long* acc2;
    unsigned long long* wide2;
    long long* acc8;
    double* accf;
    const double2* tw;
    const float2* twN;
    double2* P;
    double2* T;
    double* res;
    unsigned int* ticket;
};

// Decode bin k to its real value S[k] and clear it for the next period.
__device__ __forceinline__ double take_bin(const FinArgs& a, int64_t k) {
    if (a.fmt == PCAL_2BIT) {
        unsigned long long v = a.acc2[k];
        unsigned long long sl = (v & PCAL_F21_MASK) + a.wide2[k];
        unsigned long long sh = ((v >> 21) & PCAL_F21_MASK) + a.wide2[a.L + k];
        unsigned long long shl = ((v >> 42) & PCAL_F21_MASK) + a.wide2[2 * a.L + k];
        if (v) a.acc2[k] = 0;
        if (sl | sh) {
            a.wide2[k] = 0;
            a.wide2[a.L + k] = 0;
            a.wide2[2 * a.L + k] = 0;
        }
        int64_t r = k - a.a0;
        if (r < 0) r += a.L;
        double cnt = (double)(a.q + (r < a.rem ? 1 : 0));
        // S = sum_c level[c]*count[c] with count[3] = shl, count[2] = sh - shl,
        // count[1] = sl - shl, count[0] = cnt - sl - sh + shl.
        return a.lev0 * cnt + a.c_l * (double)sl + a.c_h * (double)sh + a.c_hl * (double)shl;
    }
    if (a.fmt == PCAL_I8) {
        long long v = a.acc8[k];
        if (v) a.acc8[k] = 0;
        return (double)v;
    }
    double v = a.accf[k];
    if (v != 0.0) a.accf[k] = 0.0;
    return v;
}

// Warp sum with a fixed butterfly: every lane gets the same, deterministic
// value.  Needs all 32 lanes.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// K block-wide FP64 sums at once (fixed order: warp butterflies, then the
// warp totals in warp order).  blockDim.x must be a multiple of 32; sm needs
// 32*K doubles.  Every thread receives the sums.
template <int K>
__device__ void block_sums(double (&v)[K], double* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = warp_sum(v[j]);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < K; ++j) sm[warp * K + j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sm[w * K + j];
        v[j] = s;
    }
    __syncthreads();
}

// Exclusive block-wide prefix sum (fixed order), any multiple of 32 threads.
__device__ double block_exclusive_scan(double v, double* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    double before = 0.0;
    for (int w = 0; w < warp; ++w) before += sm[w];
    __syncthreads();
    return before + inc - v;
}

__device__ __forceinline__ double wrap_pi(double x) {
    // into [-pi, pi)
    const double two_pi = 6.283185307179586476925, inv = 0.159154943091895335769;
    return x - two_pi * floor((x + 3.141592653589793238463) * inv);
}

// Tones [i0, i1) of the N-point DFT of P, in FP32; P is staged in shared
// memory as float2.  Groups of g threads (a power of two <= 32) share a
// tone and combine their partial sums with a fixed butterfly.
__device__ void dft_tones(const FinArgs& a, int64_t i0, int64_t i1, float2* sP) {
    const int64_t N = a.N;
    for (int64_t b = threadIdx.x; b < N; b += blockDim.x) {
        double2 v = __ldcg(&a.P[b]);
        sP[b] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    const int64_t ntone = i1 - i0;
    int g = 1;
    while (g < 32 && (int64_t)(g * 2) * ntone <= (int64_t)blockDim.x) g *= 2;
    const int groups = blockDim.x / g;
    const int sub = threadIdx.x % g;
    for (int64_t base = 0; base < ntone; base += groups) {
        const int64_t i = i0 + base + threadIdx.x / g;
        float re = 0.f, im = 0.f;
        if (i < i1) {
            int64_t idx = (i * sub) % N;
            const int64_t step = (i * g) % N;
            for (int64_t b = sub; b < N; b += g) {
                const float2 p = sP[b];
                const float2 w = a.twN[idx];
                re = fmaf(p.x, w.x, fmaf(-p.y, w.y, re));
                im = fmaf(p.x, w.y, fmaf(p.y, w.x, im));
                idx += step;
                if (idx >= N) idx -= N;
            }
        }
        for (int o = g / 2; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (i < i1 && sub == 0) a.T[i] = make_double2((double)re, (double)im);
    }
}

// Amplitude, phase, unwrapped phase and the weighted LS delay fit over all N
// tones; run by one CTA after every T_i is in global memory.
__device__ void tone_products(const FinArgs& a, double* sm) {
    const int64_t N = a.N;
    const int nt = blockDim.x, t = threadIdx.x;
    const int64_t chunk = (N + nt - 1) / nt;
    const int64_t c0 = t * chunk < N ? t * chunk : N;
    const int64_t c1 = c0 + chunk < N ? c0 + chunk : N;
    double* amp = a.res + 2 * N;
    double* ph = a.res + 3 * N;
    double* un = a.res + 4 * N;
    const double two_over_m = a.M > 0 ? 2.0 / a.M : 0.0;
    // 1. per tone
    for (int64_t i = c0; i < c1; ++i) {
        double2 z = __ldcg(&a.T[i]);
        a.res[2 * i] = z.x;
        a.res[2 * i + 1] = z.y;
        amp[i] = sqrt(z.x * z.x + z.y * z.y) * two_over_m;
        double psi = (double)atan2f((float)z.y, (float)z.x) + 1.570796326794896619231;
        ph[i] = wrap_pi(psi);
    }
    __syncthreads();
    // 2. unwrap: u_i = psi_0 + sum_{j=1..i} wrap(psi_j - psi_{j-1})
    double local = 0.0;
    for (int64_t i = c0; i < c1; ++i)
        if (i > 0) local += wrap_pi(ph[i] - ph[i - 1]);
    double run = ph[0] + block_exclusive_scan(local, sm);
    for (int64_t i = c0; i < c1; ++i) {
        if (i > 0) run += wrap_pi(ph[i] - ph[i - 1]);
        un[i] = run;
    }
    __syncthreads();
    // 3. weighted least squares of un[i] against f_i with w_i = |T_i|^2
    double s3[3] = {0.0, 0.0, 0.0};
    for (int64_t i = c0; i < c1; ++i) {
        const double w = a.res[2 * i] * a.res[2 * i] + a.res[2 * i + 1] * a.res[2 * i + 1];
        s3[0] += w;
        s3[1] += w * ((double)i * a.fc + a.fo);
        s3[2] += w * un[i];
    }
    block_sums<3>(s3, sm);
    const double W = s3[0];
    double td = nan(""), sig = nan("");
    if (N >= 2 && W > 0) {
        const double fbar = s3[1] / W, ubar = s3[2] / W;
        double s2[2] = {0.0, 0.0};
        for (int64_t i = c0; i < c1; ++i) {
            const double w = a.res[2 * i] * a.res[2 * i] + a.res[2 * i + 1] * a.res[2 * i + 1];
            const double df = (double)i * a.fc + a.fo - fbar;
            s2[0] += w * df * df;
            s2[1] += w * df * (un[i] - ubar);
        }
        block_sums<2>(s2, sm);
        if (s2[0] > 0) {
            const double slope = s2[1] / s2[0];
            double s1[1] = {0.0};
            for (int64_t i = c0; i < c1; ++i) {
                const double w = a.res[2 * i] * a.res[2 * i] + a.res[2 * i + 1] * a.res[2 * i + 1];
                const double r = un[i] - ubar - slope * ((double)i * a.fc + a.fo - fbar);
                s1[0] += w * r * r;
            }
            block_sums<1>(s1, sm);
            td = slope / 6.283185307179586476925;
            if (N > 2) sig = sqrt((s1[0] / (double)(N - 2)) / s2[0]) / 6.283185307179586476925;
        }
    }
    if (t == 0) {
        a.res[5 * N] = td;
        a.res[5 * N + 1] = sig;
        a.res[5 * N + 2] = a.M;
    }
}

// Decode + FP64 rotation + fold of whole residues; the last CTA continues.
// Thread t works on residue b = blockIdx.x*bc + t/tpb and bins b + m*N for
// m = t%tpb, t%tpb + tpb, ...; the tpb threads of a residue are contiguous
// (tpb a power of two) and combine with shuffles, then across warps.
__global__ void fin_fold_kernel(FinArgs a) {
    extern __shared__ double2 smem2[];
    __shared__ bool is_last;
    const int tpb = a.tpb;
    const int bl = threadIdx.x / tpb, sub = threadIdx.x % tpb;
    const int64_t b = (int64_t)blockIdx.x * a.bc + bl;
    const bool active = bl < a.bc && b < a.N;
    const int64_t per = a.L / a.N;
    double re = 0.0, im = 0.0;
    if (active) {
        for (int64_t m = sub; m < per; m += tpb) {
            const int64_t k = b + m * a.N;
            const double S = take_bin(a, k);
            const double2 w = a.tw[(a.so * k) % a.L];
            re = fma(S, w.x, re);
            im = fma(S, w.y, im);
        }
    }
    const int width = tpb < 32 ? tpb : 32;
    for (int o = width / 2; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (tpb <= 32) {
        if (active && sub == 0) a.P[b] = make_double2(re, im);
    } else {
        double2* wsum = smem2;
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = make_double2(re, im);
        __syncthreads();
        if (active && sub == 0) {
            double sr = 0.0, si = 0.0;
            const int w0 = threadIdx.x >> 5;
            for (int w = 0; w < tpb / 32; ++w) {
                sr += wsum[w0 + w].x;
                si += wsum[w0 + w].y;
            }
            a.P[b] = make_double2(sr, si);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&a.ticket[0], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ticket[0] = 0;
    if (a.N <= kDftInFoldMaxN) {
        dft_tones(a, 0, a.N, reinterpret_cast<float2*>(smem2 + blockDim.x));
        __threadfence();
        __syncthreads();
        tone_products(a, reinterpret_cast<double*>(smem2));
    }
}

// Spread DFT for large N; the last CTA runs the products.
__global__ void fin_dft_kernel(FinArgs a) {
    extern __shared__ double2 smem2[];
    __shared__ bool is_last;
    const int64_t i0 = (int64_t)blockIdx.x * kDftTonesPerCta;
    const int64_t i1 = i0 + kDftTonesPerCta < a.N ? i0 + kDftTonesPerCta : a.N;
    dft_tones(a, i0, i1, reinterpret_cast<float2*>(smem2 + blockDim.x));
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&a.ticket[1], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ticket[1] = 0;
    tone_products(a, reinterpret_cast<double*>(smem2));
}

__global__ void init_twiddles_kernel(double2* tw, int64_t L, float2* twN, int64_t N, int64_t sc) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < L; m += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)L, &s, &c);
        tw[m] = make_double2(c, -s);
        if (m % sc == 0 && m / sc < N) twN[m / sc] = make_float2((float)c, (float)-s);
    }
}

}  // namespace

cudaError_t launch_init_twiddles(pcal_plan* p, cudaStream_t s) {
    int64_t L = p->g.L;
    int g = (int)((L + 255) / 256);
    if (g > p->num_sms * 8) g = p->num_sms * 8;
    init_twiddles_kernel<<<g, 256, 0, s>>>(p->d_tw, L, p->d_twN, p->g.N, p->g.step_comb);
    p->stats.kernel_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_finalize(pcal_plan* p, cudaStream_t s) {
    FinArgs a{};
    const pcal_geometry& g = p->g;
    a.fmt = g.format;
    a.L = g.L;
    a.N = g.N;
    a.so = g.step_offset;
    const int64_t n_tot = p->n_abs - p->period_start;
    a.q = n_tot / g.L;
    a.rem = n_tot % g.L;
    a.a0 = p->period_start % g.L;
    const double* lv = p->levels;
    a.lev0 = lv[0];
    a.c_l = lv[1] - lv[0];
    a.c_h = lv[2] - lv[0];
    a.c_hl = lv[3] - lv[2] - lv[1] + lv[0];
    a.M = (double)n_tot;
    a.fc = (double)g.f_comb;
    a.fo = (double)g.f_offset;
    a.acc2 = p->d_acc2;
    a.wide2 = p->d_wide2;
    a.acc8 = p->d_acc8;
    a.accf = p->d_accf;
    a.tw = p->d_tw;
    a.twN = p->d_twN;
    a.P = p->d_P;
    a.T = p->d_T;
    a.res = p->d_res;
    a.ticket = p->d_ticket;

    int G = (int)(g.N < p->num_sms ? g.N : p->num_sms);
    a.bc = (int)((g.N + G - 1) / G);
    G = (int)((g.N + a.bc - 1) / a.bc);
    // tpb = the largest power of two with bc*tpb <= 256; the block is a
    // multiple of 32 threads (the shuffles and the DFT need whole warps)
    a.tpb = 1;
    while (a.bc * a.tpb * 2 <= 256) a.tpb *= 2;
    int threads = (a.bc * a.tpb + 31) / 32 * 32;
    size_t smem = (size_t)threads * sizeof(double2);
    if (g.N <= kDftInFoldMaxN) smem += (size_t)g.N * sizeof(float2);
    cudaError_t e = cudaSuccess;
    static size_t fold_smem_set = 0;
    if (smem > fold_smem_set) {
        e = cudaFuncSetAttribute(fin_fold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fold_smem_set = smem;
    }
    fin_fold_kernel<<<G, threads, smem, s>>>(a);
    p->stats.kernel_launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess || g.N <= kDftInFoldMaxN) return e;
    const int threads2 = 256;
    const size_t smem2 = threads2 * sizeof(double2) + (size_t)g.N * sizeof(float2);
    static size_t dft_smem_set = 0;
    if (smem2 > dft_smem_set) {
        e = cudaFuncSetAttribute(fin_dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        if (e != cudaSuccess) return e;
        dft_smem_set = smem2;
    }
    fin_dft_kernel<<<(unsigned)((g.N + kDftTonesPerCta - 1) / kDftTonesPerCta), threads2, smem2, s>>>(a);
    p->stats.kernel_launches += 1;
    return cudaGetLastError();
}
