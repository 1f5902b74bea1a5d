// Finalize kernels of libpcal: from the L accumulated bins to N tone phasors
// and the delay (paper Sec. 2).
//
//   decode   S[k] from the exact bins (2-bit: the level table applied to the
//            per-code counts; int8/float32: the sums)                 FP64
//   rotate   R[k] = S[k] * exp(-j*2*pi*f_offset*k/fs)        (Eq. 3)  FP64
//   fold     P[b] = sum_m R[b + m*N]                          (Eq. 2)  FP64
//            per thread, then double-float (df) across threads
//   DFT      T_i = sum_b P[b] exp(-j*2*pi*i*b/N)   (DFT(P), Sec. 2)   FP32
//   products amp_i = 2|T_i|/M and phase arg(T_i)+pi/2 (sin model of Eq. 1)
//            in FP32; the phase unwrapped along the comb and the delay as
//            the |T|^2-weighted least-squares slope of phase versus tone
//            frequency (phi_i = 2*pi*f_i*t_d, Eq. 1) in df.
//
// The rotator phase is reduced exactly in integers, (f_offset/g * k) mod L,
// and looked up in the plan's FP64 table exp(-j*2*pi*m/L) (the precomputed
// rotator of Sec. 2 after Eq. 4, built once per plan).  GB300 runs FP64 at
// about 1/64 of its FP32 rate, so FP64 stops after the per-bin rotation;
// every sum over many terms after that uses df (see df64.cuh), which keeps
// about 48 bits with FP32 instructions.
//
// Work split: the fold kernel gives each CTA whole residues b (no two CTAs
// add into the same P[b]); the last CTA to finish (an atomic ticket, no
// waiting) runs the DFT for small N and the products.  For large N a second
// kernel spreads the DFT over CTAs and its last CTA runs the products.
#include <math.h>

#include "df64.cuh"
#include "internal.cuh"

namespace {

using pcal_df::df;

constexpr int kDftInFoldMaxN = 256;
constexpr int kDftTonesPerCta = 32;

struct FinArgs {
    int fmt;
    int bc;   // residues b per fold CTA
    int tpb;  // threads per residue (power of two)
    int64_t L, N, so;
    int64_t q, rem, a0;  // samples in bin k: q + ((k - a0) mod L < rem)
    double lev0, c_l, c_h, c_hl;
    double M;
    float two_over_m;
    df two_pi_fc;  // 2*pi*f_comb in df
    unsigned long long* acc2;
    unsigned long long* wide2;
    long long* acc8;
    float2* accf;  // float32 bins in df (hi, lo)
    const double2* tw;
    const float2* twN;
    float4* P;     // P[b] as df re (x, y), df im (z, w)
    float2* T;     // FP32 tone phasors
    double* res;
    unsigned int* ticket;
};

// Decode bin k to its real value S[k] (FP64) and clear it for the next period.
__device__ __forceinline__ double take_bin(const FinArgs& a, int64_t k) {
    if (a.fmt == PCAL_2BIT) {
        const unsigned long long v = a.acc2[k];
        const unsigned long long sl = (v & PCAL_F21_MASK) + a.wide2[k];
        const unsigned long long sh = ((v >> 21) & PCAL_F21_MASK) + a.wide2[a.L + k];
        const unsigned long long shl = ((v >> 42) & PCAL_F21_MASK) + a.wide2[2 * a.L + k];
        if (v) a.acc2[k] = 0;
        if (sl | sh) {
            a.wide2[k] = 0;
            a.wide2[a.L + k] = 0;
            a.wide2[2 * a.L + k] = 0;
        }
        int64_t r = k - a.a0;
        if (r < 0) r += a.L;
        const double cnt = (double)(a.q + (r < a.rem ? 1 : 0));
        // S = sum_c level[c]*count[c] with count[3] = shl, count[2] = sh - shl,
        // count[1] = sl - shl, count[0] = cnt - sl - sh + shl.
        return a.lev0 * cnt + a.c_l * (double)sl + a.c_h * (double)sh + a.c_hl * (double)shl;
    }
    if (a.fmt == PCAL_I8) {
        const long long v = a.acc8[k];
        if (v) a.acc8[k] = 0;
        return (double)v;
    }
    const float2 v = a.accf[k];
    a.accf[k] = make_float2(0.f, 0.f);
    return (double)v.x + (double)v.y;
}

__device__ __forceinline__ df df_of(double x) {
    const float hi = (float)x;
    return df{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ df shfl_xor_df(df v, int o) {
    return df{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// K block-wide df sums (fixed order: warp butterflies, then warp totals in
// warp order); every thread receives them.  blockDim.x: a multiple of 32;
// sm: 32*K float2.
template <int K>
__device__ void block_sums_df(df (&v)[K], float2* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] = pcal_df::add(v[j], shfl_xor_df(v[j], o));
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < K; ++j) sm[warp * K + j] = make_float2(v[j].hi, v[j].lo);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) {
        df s{0.f, 0.f};
        for (int w = 0; w < nw; ++w) s = pcal_df::add(s, df{sm[w * K + j].x, sm[w * K + j].y});
        v[j] = s;
    }
    __syncthreads();
}

// Exclusive block-wide df prefix sum (fixed order).
__device__ df block_exclusive_scan_df(df v, float2* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    df inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const df u{__shfl_up_sync(0xffffffffu, inc.hi, o), __shfl_up_sync(0xffffffffu, inc.lo, o)};
        if (lane >= o) inc = pcal_df::add(inc, u);
    }
    if (lane == 31) sm[warp] = make_float2(inc.hi, inc.lo);
    __syncthreads();
    df before{0.f, 0.f};
    for (int w = 0; w < warp; ++w) before = pcal_df::add(before, df{sm[w].x, sm[w].y});
    __syncthreads();
    return pcal_df::sub(pcal_df::add(before, inc), v);
}

__device__ __forceinline__ float wrap_pi_f(float x) {
    // into [-pi, pi)
    return x - 6.283185307179586f * floorf((x + 3.141592653589793f) * 0.15915494309189535f);
}

// Tones [i0, i1) of the N-point DFT of P, in FP32.  Groups of g threads (a
// power of two <= 32) share a tone and combine their partial sums with a
// fixed butterfly.
__device__ void dft_tones(const FinArgs& a, int64_t i0, int64_t i1, float2* sP) {
    const int64_t N = a.N;
    for (int64_t b = threadIdx.x; b < N; b += blockDim.x) {
        const float4 v = __ldcg(&a.P[b]);
        sP[b] = make_float2(v.x + v.y, v.z + v.w);
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
        if (i < i1 && sub == 0) a.T[i] = make_float2(re, im);
    }
    __syncthreads();
}

// Shared memory of tone_products: psi[N] floats, un[N] float2, then 96
// float2 of reduction scratch.
__host__ __device__ size_t products_smem(int64_t N) {
    return (size_t)((N * 4 + 15) / 16) * 16 + (size_t)N * 8 + 96 * 8;
}

// Amplitude, phase, unwrapped phase and the weighted LS delay fit over all N
// tones; one CTA, after every T_i is in global memory.
__device__ void tone_products(const FinArgs& a, uint8_t* smem) {
    const int64_t N = a.N;
    const int nt = blockDim.x, t = threadIdx.x;
    float* psi = reinterpret_cast<float*>(smem);
    float2* un = reinterpret_cast<float2*>(smem + ((N * 4 + 15) / 16) * 16);
    float2* red = un + N;
    const int64_t chunk = (N + nt - 1) / nt;
    const int64_t c0 = t * chunk < N ? t * chunk : N;
    const int64_t c1 = c0 + chunk < N ? c0 + chunk : N;
    double* amp = a.res + 2 * N;
    double* ph = a.res + 3 * N;
    double* unw = a.res + 4 * N;
    // 1. per tone, FP32
    for (int64_t i = c0; i < c1; ++i) {
        const float2 z = __ldcg(&a.T[i]);
        const float p = wrap_pi_f(atan2f(z.y, z.x) + 1.5707963267948966f);
        psi[i] = p;
        a.res[2 * i] = (double)z.x;
        a.res[2 * i + 1] = (double)z.y;
        amp[i] = (double)(sqrtf(z.x * z.x + z.y * z.y) * a.two_over_m);
        ph[i] = (double)p;
    }
    __syncthreads();
    // 2. unwrap: u_i = psi_0 + sum_{j=1..i} wrap(psi_j - psi_{j-1}), df sums
    df local{0.f, 0.f};
    for (int64_t i = c0; i < c1; ++i)
        if (i > 0) local = pcal_df::add_f(local, wrap_pi_f(psi[i] - psi[i - 1]));
    df run = pcal_df::add_f(block_exclusive_scan_df(local, red), psi[0]);
    for (int64_t i = c0; i < c1; ++i) {
        if (i > 0) run = pcal_df::add_f(run, wrap_pi_f(psi[i] - psi[i - 1]));
        un[i] = make_float2(run.hi, run.lo);
        unw[i] = (double)run.hi + (double)run.lo;
    }
    __syncthreads();
    // 3. weighted least squares of u_i against the tone index x_i = i (the
    //    frequency is f_i = f_comb*i + f_offset), weights w_i = |T_i|^2
    df s3[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int64_t i = c0; i < c1; ++i) {
        const float2 z = __ldcg(&a.T[i]);
        const float w = z.x * z.x + z.y * z.y;
        s3[0] = pcal_df::add_f(s3[0], w);
        s3[1] = pcal_df::add(s3[1], pcal_df::two_prod(w, (float)i));
        s3[2] = pcal_df::add(s3[2], pcal_df::mul_f(df{un[i].x, un[i].y}, w));
    }
    block_sums_df<3>(s3, red);
    const df W = s3[0];
    double td = nan(""), sig = nan("");
    if (N >= 2 && W.hi > 0.f) {
        const df xbar = pcal_df::div(s3[1], W), ubar = pcal_df::div(s3[2], W);
        df s2[2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (int64_t i = c0; i < c1; ++i) {
            const float2 z = __ldcg(&a.T[i]);
            const float w = z.x * z.x + z.y * z.y;
            const df dx = pcal_df::sub(df{(float)i, 0.f}, xbar);
            const df du = pcal_df::sub(df{un[i].x, un[i].y}, ubar);
            const df wdx = pcal_df::mul_f(dx, w);
            s2[0] = pcal_df::add(s2[0], pcal_df::mul(wdx, dx));
            s2[1] = pcal_df::add(s2[1], pcal_df::mul(wdx, du));
        }
        block_sums_df<2>(s2, red);
        if (s2[0].hi > 0.f) {
            const df slope = pcal_df::div(s2[1], s2[0]);  // rad per tone index
            df s1[1] = {{0.f, 0.f}};
            for (int64_t i = c0; i < c1; ++i) {
                const float2 z = __ldcg(&a.T[i]);
                const float w = z.x * z.x + z.y * z.y;
                const df dx = pcal_df::sub(df{(float)i, 0.f}, xbar);
                const df r = pcal_df::sub(pcal_df::sub(df{un[i].x, un[i].y}, ubar), pcal_df::mul(slope, dx));
                s1[0] = pcal_df::add(s1[0], pcal_df::mul_f(pcal_df::mul(r, r), w));
            }
            block_sums_df<1>(s1, red);
            const df tdd = pcal_df::div(slope, a.two_pi_fc);
            td = (double)tdd.hi + (double)tdd.lo;
            if (N > 2) {
                const df v = pcal_df::div(pcal_df::div(s1[0], df{(float)(N - 2), 0.f}), s2[0]);
                const df sd = pcal_df::div(pcal_df::sqrt_df(v), a.two_pi_fc);
                sig = (double)sd.hi + (double)sd.lo;
            }
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
    extern __shared__ __align__(16) uint8_t smem[];
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
    df dre = df_of(re), dim = df_of(im);
    const int width = tpb < 32 ? tpb : 32;
    for (int o = width / 2; o > 0; o >>= 1) {
        dre = pcal_df::add(dre, shfl_xor_df(dre, o));
        dim = pcal_df::add(dim, shfl_xor_df(dim, o));
    }
    if (tpb <= 32) {
        if (active && sub == 0) a.P[b] = make_float4(dre.hi, dre.lo, dim.hi, dim.lo);
    } else {
        float4* wsum = reinterpret_cast<float4*>(smem);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = make_float4(dre.hi, dre.lo, dim.hi, dim.lo);
        __syncthreads();
        if (active && sub == 0) {
            df sr{0.f, 0.f}, si{0.f, 0.f};
            const int w0 = threadIdx.x >> 5;
            for (int w = 0; w < tpb / 32; ++w) {
                const float4 v = wsum[w0 + w];
                sr = pcal_df::add(sr, df{v.x, v.y});
                si = pcal_df::add(si, df{v.z, v.w});
            }
            a.P[b] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
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
        dft_tones(a, 0, a.N, reinterpret_cast<float2*>(smem));
        __threadfence();
        tone_products(a, smem);
    }
}

// Spread DFT for large N; the last CTA runs the products.
__global__ void fin_dft_kernel(FinArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ bool is_last;
    const int64_t i0 = (int64_t)blockIdx.x * kDftTonesPerCta;
    const int64_t i1 = i0 + kDftTonesPerCta < a.N ? i0 + kDftTonesPerCta : a.N;
    dft_tones(a, i0, i1, reinterpret_cast<float2*>(smem));
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&a.ticket[1], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ticket[1] = 0;
    tone_products(a, smem);
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
    a.two_over_m = n_tot > 0 ? (float)(2.0 / (double)n_tot) : 0.0f;
    const double tpf = 6.283185307179586476925 * (double)g.f_comb;
    a.two_pi_fc.hi = (float)tpf;
    a.two_pi_fc.lo = (float)(tpf - (double)a.two_pi_fc.hi);
    a.acc2 = p->d_acc2;
    a.wide2 = p->d_wide2;
    a.acc8 = p->d_acc8;
    a.accf = p->d_accf;
    a.tw = p->d_tw;
    a.twN = p->d_twN;
    a.P = reinterpret_cast<float4*>(p->d_P);
    a.T = reinterpret_cast<float2*>(p->d_T);
    a.res = p->d_res;
    a.ticket = p->d_ticket;

    int G = (int)(g.N < p->num_sms ? g.N : p->num_sms);
    a.bc = (int)((g.N + G - 1) / G);
    G = (int)((g.N + a.bc - 1) / a.bc);
    // tpb = the largest power of two with bc*tpb <= 256; the block is a
    // multiple of 32 threads (the shuffles and the DFT need whole warps)
    a.tpb = 1;
    while (a.bc * a.tpb * 2 <= 256) a.tpb *= 2;
    const int threads = (a.bc * a.tpb + 31) / 32 * 32;
    size_t smem = (size_t)threads * 16;
    if (g.N <= kDftInFoldMaxN) {
        const size_t need = products_smem(g.N) > (size_t)g.N * 8 ? products_smem(g.N) : (size_t)g.N * 8;
        if (need > smem) smem = need;
    }
    cudaError_t e = cudaSuccess;
    static size_t fold_smem_set = 0;
    if (smem > 48 * 1024 && smem > fold_smem_set) {
        e = cudaFuncSetAttribute(fin_fold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fold_smem_set = smem;
    }
    fin_fold_kernel<<<G, threads, smem, s>>>(a);
    p->stats.kernel_launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess || g.N <= kDftInFoldMaxN) return e;
    const int threads2 = 256;
    const size_t smem2 = (size_t)g.N * 8 > products_smem(g.N) ? (size_t)g.N * 8 : products_smem(g.N);
    static size_t dft_smem_set = 0;
    if (smem2 > 48 * 1024 && smem2 > dft_smem_set) {
        e = cudaFuncSetAttribute(fin_dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        if (e != cudaSuccess) return e;
        dft_smem_set = smem2;
    }
    fin_dft_kernel<<<(unsigned)((g.N + kDftTonesPerCta - 1) / kDftTonesPerCta), threads2, smem2, s>>>(a);
    p->stats.kernel_launches += 1;
    return cudaGetLastError();
}
