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
// Work split.  For N <= 256 and L <= 32768 (every plan of the benchmark
// workloads) one thread-block cluster does everything: each CTA folds a
// slice of the bins into a partial P, the partials meet in distributed
// shared memory, and CTA 0 runs the DFT from shared memory and the products
// in one warp, so no result makes a round trip through global memory.
// Otherwise the fold kernel gives each CTA whole residues b (no two CTAs add
// into the same P[b]); the last CTA to finish (an atomic ticket, no waiting)
// runs the DFT for small N and the products.  For large N a second kernel
// spreads the DFT over CTAs and its last CTA runs the products.
#include <cooperative_groups.h>
#include <math.h>

#include <mutex>

#include "df64.cuh"
#include "internal.cuh"

namespace {

using pcal_df::df;

constexpr int kDftInFoldMaxN = 256;
constexpr int kDftTonesPerCta = 32;

struct FinArgs {
    int fmt;
    int spilled;  // 2-bit: the wide arrays hold counts of this period
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
    // float32: fold partials not yet added into accf (slot e: [pf_rg[e]][pf_cols], column 0 = bin pf_ka[e])
    const float2* pf[kPartSlots];
    int64_t pf_rg[kPartSlots];
    int64_t pf_ka[kPartSlots];
    int n_pf;
    int64_t pf_cols;
    const long long* counts4;  // no-allocation entry: the caller's counts [L][4]
    double lev[4];             // no-allocation entry: the code levels
    const double2* tw;
    const float2* twN;
    float4* P;     // P[b] as df re (x, y), df im (z, w)
    float2* T;     // FP32 tone phasors
    double* res;
    double* extra;  // post-processing, N+2 doubles (or null): peak delay, peak position, corrected bandpass phase
    float2* Pout;   // cluster finalize: if set, store P here and stop before the DFT
    double fs_hz;
    unsigned int* ticket;
};

// Decode bin k to its real value S[k] (FP64).  NoAlloc: the caller's
// per-(bin, code) counts.
template <bool NoAlloc, int FMT = -1>
__device__ __forceinline__ double read_bin(const FinArgs& a, int64_t k) {
    const int fmt = FMT < 0 ? a.fmt : FMT;
    if constexpr (NoAlloc) {
        const long long* c = a.counts4 + 4 * k;
        return a.lev[0] * (double)c[0] + a.lev[1] * (double)c[1] + a.lev[2] * (double)c[2] + a.lev[3] * (double)c[3];
    }
    if (fmt == PCAL_2BIT) {
        const unsigned long long v = a.acc2[k];
        unsigned long long sl = v & PCAL_F21_MASK, sh = (v >> 21) & PCAL_F21_MASK, shl = (v >> 42) & PCAL_F21_MASK;
        if (a.spilled) {
            sl += a.wide2[k];
            sh += a.wide2[a.L + k];
            shl += a.wide2[2 * a.L + k];
        }
        int64_t r = k - a.a0;
        if (r < 0) r += a.L;
        const double cnt = (double)(a.q + (r < a.rem ? 1 : 0));
        // S = sum_c level[c]*count[c] with count[3] = shl, count[2] = sh - shl,
        // count[1] = sl - shl, count[0] = cnt - sl - sh + shl.
        return a.lev0 * cnt + a.c_l * (double)sl + a.c_h * (double)sh + a.c_hl * (double)shl;
    }
    if (fmt == PCAL_I8) return (double)a.acc8[k];
    const float2 v = a.accf[k];
    if (a.n_pf == 0) return (double)v.x + (double)v.y;
    // the pending fold partials of this bin, slot by slot, row group by row
    // group, in double-float (a fixed order: the result does not depend on
    // timing).  Inline: out of line (a call per bin) the C1 step took
    // 1.5 us longer.
    df s{v.x, v.y};
    for (int e = 0; e < a.n_pf; ++e) {
        const int64_t R = a.pf_rg[e], stride = a.pf_cols;
        for (int64_t c = ((k - a.pf_ka[e]) % a.L + a.L) % a.L; c < a.pf_cols; c += a.L) {
            const float2* col = a.pf[e] + c;
            int64_t rg = 0;
            // eight loads in flight, then their additions in row-group order
            for (; rg + 8 <= R; rg += 8) {
                float2 w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) w[u] = col[(rg + u) * stride];
#pragma unroll
                for (int u = 0; u < 8; ++u) s = pcal_df::add(s, pcal_df::two_sum(w[u].x, w[u].y));
            }
            for (; rg < R; ++rg) {
                const float2 w = col[rg * stride];
                s = pcal_df::add(s, pcal_df::two_sum(w.x, w.y));
            }
        }
    }
    return (double)s.hi + (double)s.lo;
}

// exp(-j*2*pi*m/L): the plan's table; NoAlloc evaluates it here.
template <bool NoAlloc>
__device__ __forceinline__ double2 rotator(const FinArgs& a, int64_t m) {
    if constexpr (NoAlloc) {
        double sn, cs;
        sincospi(2.0 * (double)m / (double)a.L, &sn, &cs);
        return make_double2(cs, -sn);
    }
    return a.tw[m];
}

// Clear bin k for the next integration period.
// FMT: the plan's sample format where the kernel is specialised for one
// (its other formats' code is left out), or -1 for the run-time a.fmt.
template <int FMT = -1>
__device__ __forceinline__ void clear_bin(const FinArgs& a, int64_t k) {
    const int fmt = FMT < 0 ? a.fmt : FMT;
    if (fmt == PCAL_2BIT) {
        a.acc2[k] = 0;
        if (a.spilled) {
            a.wide2[k] = 0;
            a.wide2[a.L + k] = 0;
            a.wide2[2 * a.L + k] = 0;
        }
    } else if (fmt == PCAL_I8) {
        a.acc8[k] = 0;
    } else {
        a.accf[k] = make_float2(0.f, 0.f);
    }
}

// Programmatic dependent launch: wait for the preceding kernel's results;
// allow the following kernel to start launching.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Completion ticket: a release-acquire increment, so the arriving CTA's
// stores are visible to the CTA that draws the last ticket.
__device__ __forceinline__ unsigned int ticket_acq_rel(unsigned int* t) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(t) : "memory");
    return old;
}

__device__ __forceinline__ df df_of(double x) {
    const float hi = (float)x;
    return df{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ df shfl_xor_df(df v, int o) {
    return df{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// K block-wide df sums (fixed order: warp butterflies, then the totals of
// the first nw warps in warp order -- the other warps hold zeros); every
// thread receives them.  blockDim.x: a multiple of 32; sm: 32*K float2.
template <int K>
__device__ void block_sums_df(df (&v)[K], float2* sm, int nw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] = pcal_df::add(v[j], shfl_xor_df(v[j], o));
    if (nw == 1) {
        __syncthreads();  // keep the barrier count equal for every nw
        return;
    }
    if (lane == 0 && warp < nw)
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

// Tones [i0, i1) of the N-point DFT of P, in FP32, written to global T and,
// when sT is given, to shared memory.  P (hi + lo) and the twiddles are
// staged in shared memory first.  Groups of g threads (a power of two <= 32)
// share a tone and combine their partial sums with a fixed butterfly.
template <bool NoAlloc>
__device__ void dft_tones(const FinArgs& a, int64_t i0, int64_t i1, float2* sP, float2* sTw, float2* sT) {
    const int64_t N = a.N;
    for (int64_t b = threadIdx.x; b < N; b += blockDim.x) {
        const float4 v = __ldcg(&a.P[b]);
        sP[b] = make_float2(v.x + v.y, v.z + v.w);
        if constexpr (NoAlloc) {
            float sn, cs;
            sincospif(2.0f * (float)b / (float)N, &sn, &cs);
            sTw[b] = make_float2(cs, -sn);
        } else {
            sTw[b] = a.twN[b];
        }
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
            int idx = (int)((i * sub) % N);
            const int step = (int)((i * g) % N);
            const int n = (int)N;
            for (int b = sub; b < n; b += g) {
                const float2 p = sP[b];
                const float2 w = sTw[idx];
                re = fmaf(p.x, w.x, fmaf(-p.y, w.y, re));
                im = fmaf(p.x, w.y, fmaf(p.y, w.x, im));
                idx += step;
                if (idx >= n) idx -= n;
            }
        }
        for (int o = g / 2; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (i < i1 && sub == 0) {
            a.T[i] = make_float2(re, im);
            if (sT) sT[i] = make_float2(re, im);
        }
    }
    __syncthreads();
}

// Shared memory of the products: T[N] float2, psi[N] float, un[N] float2,
// then reduction scratch (96 float2) and the two df results.
struct ProductsSmem {
    float2* T;
    float* psi;
    float2* un;
    float2* red;
    float2* out;  // [0] td (df), [1] sigma (df)
};

__host__ __device__ inline size_t products_bytes(int64_t N) {
    return (size_t)N * 8 + (size_t)((N * 4 + 15) / 16) * 16 + (size_t)N * 8 + 98 * 8;
}

__device__ inline ProductsSmem products_layout(uint8_t* base, int64_t N) {
    ProductsSmem m;
    m.T = reinterpret_cast<float2*>(base);
    m.psi = reinterpret_cast<float*>(base + N * 8);
    m.un = reinterpret_cast<float2*>(base + N * 8 + ((N * 4 + 15) / 16) * 16);
    m.red = m.un + N;
    m.out = m.red + 96;
    return m;
}

// Post-processing (Sec. 2, Sec. 3): the delay from the time-domain pulse --
// the largest |P[b]| and the vertex of the parabola through it and its two
// neighbours; a delay t_d puts the pulse at b = -t_d*fs (mod N) -- into
// extra[0] (seconds, wrapped into one comb period) and extra[1] (the peak
// position in bins).  One warp; P is read from `P` (float2, re/im).
__device__ void peak_delay_warp(const FinArgs& a, const float2* P) {
    const int N = (int)a.N;
    const int lane = threadIdx.x & 31;
    float best = -1.f;
    int bi = 0;
#pragma unroll 1
    for (int b = lane; b < N; b += 32) {
        const float2 z = P[b];
        const float v = z.x * z.x + z.y * z.y;
        if (v > best) {
            best = v;
            bi = b;
        }
    }
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        // FP32 throughout (a position to ~1e-5 bin): scalar FP64 square roots
        // and divisions are long dependent chains on GB300's FP64 pipe
        const float2 zm = P[(bi + N - 1) % N], zp = P[(bi + 1) % N];
        const float ym = sqrtf(zm.x * zm.x + zm.y * zm.y), y0 = sqrtf(best);
        const float yp = sqrtf(zp.x * zp.x + zp.y * zp.y);
        const float den = ym - 2.f * y0 + yp;
        const float pos = (float)bi + (den != 0.f ? 0.5f * (ym - yp) / den : 0.f);
        // -pos wrapped into [-N/2, N/2) bins, then seconds
        float q = -pos;
        q -= (float)N * floorf((q + 0.5f * (float)N) / (float)N);
        a.extra[0] = best > 0.f ? (double)(q / (float)a.fs_hz) : __longlong_as_double(0x7ff8000000000000ll);
        a.extra[1] = (double)pos;
    }
}

// Amplitude, phase, unwrapped phase and the weighted LS delay fit over all N
// tones, from T in shared memory; one CTA.  The first nt threads (whole
// warps, about 8 tones each) do the arithmetic; all threads then write the
// FP64 results.
__device__ void tone_products(const FinArgs& a, const ProductsSmem& m) {
    const int64_t N = a.N;
    const int t = threadIdx.x;
    int nt = (int)((N + 7) / 8 + 31) / 32 * 32;
    if (nt > (int)blockDim.x) nt = blockDim.x;
    const int nw = nt / 32;  // warps holding tones
    const int64_t chunk = (N + nt - 1) / nt;
    const int64_t c0 = t < nt ? (t * chunk < N ? t * chunk : N) : N;
    const int64_t c1 = c0 + chunk < N ? c0 + chunk : N;
    // 1. phase per tone, FP32
    for (int64_t i = c0; i < c1; ++i) {
        const float2 z = m.T[i];
        m.psi[i] = wrap_pi_f(atan2f(z.y, z.x) + 1.5707963267948966f);
    }
    __syncthreads();
    // 2. unwrap: u_i = psi_0 + sum_{j=1..i} wrap(psi_j - psi_{j-1}), df sums
    df local{0.f, 0.f};
    for (int64_t i = c0; i < c1; ++i)
        if (i > 0) local = pcal_df::add_f(local, wrap_pi_f(m.psi[i] - m.psi[i - 1]));
    df run = pcal_df::add_f(block_exclusive_scan_df(local, m.red), m.psi[0]);
    for (int64_t i = c0; i < c1; ++i) {
        if (i > 0) run = pcal_df::add_f(run, wrap_pi_f(m.psi[i] - m.psi[i - 1]));
        m.un[i] = make_float2(run.hi, run.lo);
    }
    // 3. weighted least squares of u_i against the tone index x_i = i (the
    //    frequency is f_i = f_comb*i + f_offset), weights w_i = |T_i|^2
    df s3[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int64_t i = c0; i < c1; ++i) {
        const float2 z = m.T[i];
        const float w = z.x * z.x + z.y * z.y;
        s3[0] = pcal_df::add_f(s3[0], w);
        s3[1] = pcal_df::add(s3[1], pcal_df::two_prod(w, (float)i));
        s3[2] = pcal_df::add(s3[2], pcal_df::mul_f(df{m.un[i].x, m.un[i].y}, w));
    }
    block_sums_df<3>(s3, m.red, nw);
    const df W = s3[0];
    df td{__int_as_float(0x7fc00000), 0.f}, sig{__int_as_float(0x7fc00000), 0.f};  // NaN until fitted
    df xbar{0.f, 0.f}, ubar{0.f, 0.f}, slope{0.f, 0.f};
    bool fitted = false;
    if (N >= 2 && W.hi > 0.f) {
        xbar = pcal_df::div(s3[1], W);
        ubar = pcal_df::div(s3[2], W);
        // centred sums; the residual sum follows from Syy - slope*Sxu
        df s2[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int64_t i = c0; i < c1; ++i) {
            const float2 z = m.T[i];
            const float w = z.x * z.x + z.y * z.y;
            const df dx = pcal_df::sub(df{(float)i, 0.f}, xbar);
            const df du = pcal_df::sub(df{m.un[i].x, m.un[i].y}, ubar);
            const df wdx = pcal_df::mul_f(dx, w);
            s2[0] = pcal_df::add(s2[0], pcal_df::mul(wdx, dx));
            s2[1] = pcal_df::add(s2[1], pcal_df::mul(wdx, du));
            s2[2] = pcal_df::add(s2[2], pcal_df::mul_f(pcal_df::mul(du, du), w));
        }
        block_sums_df<3>(s2, m.red, nw);
        if (s2[0].hi > 0.f) {
            slope = pcal_df::div(s2[1], s2[0]);  // rad per tone index
            fitted = true;
            td = pcal_df::div(slope, a.two_pi_fc);
            if (N > 2) {
                df ssr = pcal_df::sub(s2[2], pcal_df::mul(slope, s2[1]));
                if (ssr.hi < 0.f) ssr = df{0.f, 0.f};
                sig = pcal_df::div(pcal_df::sqrt_df(pcal_df::div(ssr, pcal_df::mul_f(s2[0], (float)(N - 2)))),
                                   a.two_pi_fc);
            }
        }
    }
    if (t == 0) {
        m.out[0] = make_float2(td.hi, td.lo);
        m.out[1] = make_float2(sig.hi, sig.lo);
    }
    if (a.extra)  // bandpass phase with the fitted delay removed
        for (int64_t i = c0; i < c1; ++i) {
            const df r = pcal_df::sub(pcal_df::sub(df{m.un[i].x, m.un[i].y}, ubar),
                                      pcal_df::mul(slope, pcal_df::sub(df{(float)i, 0.f}, xbar)));
            a.extra[2 + i] = fitted ? (double)r.hi + (double)r.lo : __longlong_as_double(0x7ff8000000000000ll);
        }
    __syncthreads();
    // 4. FP64 results, written by all threads
    double* amp = a.res + 2 * N;
    double* ph = a.res + 3 * N;
    double* unw = a.res + 4 * N;
    for (int64_t i = t; i < N; i += blockDim.x) {
        const float2 z = m.T[i];
        a.res[2 * i] = (double)z.x;
        a.res[2 * i + 1] = (double)z.y;
        amp[i] = (double)(sqrtf(z.x * z.x + z.y * z.y) * a.two_over_m);
        ph[i] = (double)m.psi[i];
        unw[i] = (double)m.un[i].x + (double)m.un[i].y;
    }
    if (t == 0) {
        a.res[5 * N] = (double)m.out[0].x + (double)m.out[0].y;
        a.res[5 * N + 1] = (double)m.out[1].x + (double)m.out[1].y;
        a.res[5 * N + 2] = a.M;
    }
}

// Decode + FP64 rotation + fold of whole residues; the last CTA continues.
// Thread t works on residue b = blockIdx.x*bc + t/tpb and bins b + m*N for
// m = t%tpb, t%tpb + tpb, ...; the tpb threads of a residue are contiguous
// (tpb a power of two) and combine with shuffles, then across warps.
template <bool NoAlloc>
__global__ void fin_fold_kernel(FinArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ bool is_last;
    grid_dependency_wait();  // the bins of the preceding fold
    allow_dependents();
    const int tpb = a.tpb;
    const int bl = threadIdx.x / tpb, sub = threadIdx.x % tpb;
    const int64_t b = (int64_t)blockIdx.x * a.bc + bl;
    const bool active = bl < a.bc && b < a.N;
    const int64_t per = a.L / a.N;
    double re = 0.0, im = 0.0;
    if (active) {
        for (int64_t m = sub; m < per; m += tpb) {
            const int64_t k = b + m * a.N;
            const double S = read_bin<NoAlloc>(a, k);
            const double2 w = rotator<NoAlloc>(a, (a.so * k) % a.L);
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
    __threadfence();  // the P stores of this CTA's writers
    __syncthreads();
    if (threadIdx.x == 0) is_last = ticket_acq_rel(&a.ticket[0]) == gridDim.x - 1;
    // clear this CTA's bins for the next period; the fence above did not
    // have to wait for these stores
    if (!NoAlloc && active)
        for (int64_t m = sub; m < per; m += tpb) clear_bin(a, b + m * a.N);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ticket[0] = 0;
    if (a.N <= kDftInFoldMaxN) {
        // shared memory: products area, then P and the twiddles for the DFT
        const ProductsSmem m = products_layout(smem, a.N);
        float2* sP = reinterpret_cast<float2*>(smem + products_bytes(a.N));
        dft_tones<NoAlloc>(a, 0, a.N, sP, sP + a.N, m.T);
        tone_products(a, m);
        if (a.extra && threadIdx.x < 32) peak_delay_warp(a, sP);
    }
}

// ---- one-cluster finalize (N <= kClusterMaxN) ------------------------------

constexpr int kClusterMaxN = 256;       // single plans: the cluster path up to here
constexpr int kClusterBigN = 1024;      // batches: the cluster path up to here (DFT spread over the cluster)
constexpr int kClusterThreads = 256;
constexpr size_t kClusterPadSmem = 24 * 1024;
constexpr int64_t kClusterMaxL = 32768;

// Exclusive df prefix sum across the 32 lanes of a warp (fixed order).
__device__ __forceinline__ df warp_exclusive_scan_df(df v) {
    const int lane = threadIdx.x & 31;
    df inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const df u{__shfl_up_sync(0xffffffffu, inc.hi, o), __shfl_up_sync(0xffffffffu, inc.lo, o)};
        if (lane >= o) inc = pcal_df::add(inc, u);
    }
    const df prev{__shfl_up_sync(0xffffffffu, inc.hi, 1), __shfl_up_sync(0xffffffffu, inc.lo, 1)};
    return lane == 0 ? df{0.f, 0.f} : prev;
}

// K df sums over the 32 lanes by a fixed butterfly; every lane gets them.
// The steps are a loop, not unrolled: this code runs once per finalize, so
// its size (instruction fetch) costs more than its loop overhead.
template <int K>
__device__ __forceinline__ void warp_sums_df(df (&v)[K]) {
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < K; ++j) v[j] = pcal_df::add(v[j], shfl_xor_df(v[j], o));
}

// Shared memory of tone_products_warp: per tone the phase, the weight and
// the unwrapped phase (df).
struct WarpProductsSmem {
    float2* un;   // [N] unwrapped phase (df)
    float2* out;  // [2] td, sigma (df)
    float* psi;   // [N]
    float* w;     // [N]
};

// Dynamic shared memory of the cluster finalize for N tones.
struct ClusterSmem {
    float4* Pr;   // [N] this CTA's partial P (df re, df im)
    float2* sP;   // [N] P
    float2* sTw;  // [N] DFT twiddles
    float2* sT;   // [N] tone phasors
    WarpProductsSmem pm;
};

__host__ __device__ inline size_t cluster_smem_bytes(int64_t N) { return (size_t)N * 56 + 16; }

__device__ inline ClusterSmem cluster_layout(uint8_t* base, int64_t N) {
    ClusterSmem m;
    m.Pr = reinterpret_cast<float4*>(base);
    m.sP = reinterpret_cast<float2*>(base + 16 * N);
    m.sTw = m.sP + N;
    m.sT = m.sTw + N;
    m.pm.un = m.sT + N;
    m.pm.out = m.pm.un + N;
    m.pm.psi = reinterpret_cast<float*>(m.pm.out + 2);
    m.pm.w = m.pm.psi + N;
    return m;
}

// The products of tone_products, by one warp with no block barrier: lane l
// takes the contiguous tones [l*c, l*c + c), c = ceil(N/32).  Loops over a
// lane's tones are not unrolled, for the reason given at warp_sums_df.
__device__ __noinline__ void tone_products_warp(const FinArgs& a, const float2* __restrict__ sT,
                                                float* __restrict__ psi, float* __restrict__ wt,
                                                float2* __restrict__ un, float2* __restrict__ out) {
    double* const extra = a.extra;
    const int N = (int)a.N;
    const int lane = threadIdx.x & 31;
    const int c = (N + 31) / 32;
    const int i0 = lane * c < N ? lane * c : N;
    const int i1 = i0 + c < N ? i0 + c : N;
    // 1. phase and weight per tone, FP32
#pragma unroll 1
    for (int i = i0; i < i1; ++i) {
        const float2 z = sT[i];
        psi[i] = wrap_pi_f(atan2f(z.y, z.x) + 1.5707963267948966f);
        wt[i] = z.x * z.x + z.y * z.y;
    }
    __syncwarp();
    // 2. unwrap: u_i = psi_0 + sum_{j=1..i} wrap(psi_j - psi_{j-1}), df sums
    const int j0 = i0 > 1 ? i0 : 1;
    df local{0.f, 0.f};
#pragma unroll 1
    for (int i = j0; i < i1; ++i) local = pcal_df::add_f(local, wrap_pi_f(psi[i] - psi[i - 1]));
    df run = pcal_df::add_f(warp_exclusive_scan_df(local), psi[0]);
#pragma unroll 1
    for (int i = i0; i < i1; ++i) {
        if (i > 0) run = pcal_df::add_f(run, wrap_pi_f(psi[i] - psi[i - 1]));
        un[i] = make_float2(run.hi, run.lo);
    }
    // 3. weighted least squares of u_i against the tone index x_i = i (the
    //    frequency is f_i = f_comb*i + f_offset), weights w_i = |T_i|^2
    df s3[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
    for (int i = i0; i < i1; ++i) {
        const float w = wt[i];
        s3[0] = pcal_df::add_f(s3[0], w);
        s3[1] = pcal_df::add(s3[1], pcal_df::two_prod(w, (float)i));
        s3[2] = pcal_df::add(s3[2], pcal_df::mul_f(df{un[i].x, un[i].y}, w));
    }
    warp_sums_df<3>(s3);
    const df W = s3[0];
    df td{__int_as_float(0x7fc00000), 0.f}, sig{__int_as_float(0x7fc00000), 0.f};  // NaN until fitted
    df xbar{0.f, 0.f}, ubar{0.f, 0.f}, slope{0.f, 0.f};
    bool fitted = false;
    if (N >= 2 && W.hi > 0.f) {
        xbar = pcal_df::div(s3[1], W);
        ubar = pcal_df::div(s3[2], W);
        // centred sums; the residual sum follows from Syy - slope*Sxu
        df s2[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
        for (int i = i0; i < i1; ++i) {
            const float w = wt[i];
            const df dx = pcal_df::sub(df{(float)i, 0.f}, xbar);
            const df du = pcal_df::sub(df{un[i].x, un[i].y}, ubar);
            const df wdx = pcal_df::mul_f(dx, w);
            s2[0] = pcal_df::add(s2[0], pcal_df::mul(wdx, dx));
            s2[1] = pcal_df::add(s2[1], pcal_df::mul(wdx, du));
            s2[2] = pcal_df::add(s2[2], pcal_df::mul_f(pcal_df::mul(du, du), w));
        }
        warp_sums_df<3>(s2);
        if (s2[0].hi > 0.f) {
            slope = pcal_df::div(s2[1], s2[0]);  // rad per tone index
            fitted = true;
            td = pcal_df::div(slope, a.two_pi_fc);
            if (N > 2) {
                df ssr = pcal_df::sub(s2[2], pcal_df::mul(slope, s2[1]));
                if (ssr.hi < 0.f) ssr = df{0.f, 0.f};
                sig = pcal_df::div(pcal_df::sqrt_df(pcal_df::div(ssr, pcal_df::mul_f(s2[0], (float)(N - 2)))),
                                   a.two_pi_fc);
            }
        }
    }
    if (lane == 0) {
        out[0] = make_float2(td.hi, td.lo);
        out[1] = make_float2(sig.hi, sig.lo);
    }
    if (extra) {
        // bandpass phase with the fitted delay removed: u_i - ubar - slope*(i - xbar)
#pragma unroll 1
        for (int i = i0; i < i1; ++i) {
            const df r = pcal_df::sub(pcal_df::sub(df{un[i].x, un[i].y}, ubar),
                                      pcal_df::mul(slope, pcal_df::sub(df{(float)i, 0.f}, xbar)));
            extra[2 + i] = fitted ? (double)r.hi + (double)r.lo : __longlong_as_double(0x7ff8000000000000ll);
        }
    }
}

// The FP64 result vector from the products in shared memory, by the block.
__device__ void write_results_block(const FinArgs& a, const float2* sT, const WarpProductsSmem& m) {
    const int N = (int)a.N;
    double* amp = a.res + 2 * N;
    double* ph = a.res + 3 * N;
    double* unw = a.res + 4 * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float2 z = sT[i];
        a.res[2 * i] = (double)z.x;
        a.res[2 * i + 1] = (double)z.y;
        amp[i] = (double)(sqrtf(m.w[i]) * a.two_over_m);
        ph[i] = (double)m.psi[i];
        unw[i] = (double)m.un[i].x + (double)m.un[i].y;
    }
    if (threadIdx.x == 0) {
        a.res[5 * N] = (double)m.out[0].x + (double)m.out[0].y;
        a.res[5 * N + 1] = (double)m.out[1].x + (double)m.out[1].y;
        a.res[5 * N + 2] = a.M;
    }
}

// Decode, rotate (FP64, Eq. 3) and fold residue b over m = m, m + step, ...
// below m_end (bins k = b + m*N), clearing each bin; returns the FP64 sum.
template <int FMT = -1>
__device__ __forceinline__ double2 fold_residue(const FinArgs& a, int b, int m, int step, int m_end) {
    const int fmt = FMT < 0 ? a.fmt : FMT;
    double re = 0.0, im = 0.0;
    if (m >= m_end) return make_double2(0.0, 0.0);
    const int L = (int)a.L, N = (int)a.N;
    int k = b + m * N;
    int idx = (int)((a.so * k) % L);  // rotator index (f_offset/g * k) mod L
    const int kstep = step * N;
    const int istep = (int)((a.so * kstep) % L);
    if (fmt == PCAL_2BIT && !a.spilled) {
        // S = lev0*cnt + c_l*sum(l) + c_h*sum(h) + c_hl*sum(h AND l),
        // cnt = q or q + 1; the fields are below 2^21
        const double s_q = a.lev0 * (double)a.q, s_q1 = a.lev0 * (double)(a.q + 1);
        const int a0 = (int)a.a0, rem = (int)a.rem;
#pragma unroll 2
        for (; m < m_end; m += step) {
            const unsigned long long v = a.acc2[k];
            const double2 w = a.tw[idx];
            a.acc2[k] = 0;
            int rr = k - a0;
            if (rr < 0) rr += L;
            const double S = fma(a.c_hl, (double)(int)((v >> 42) & PCAL_F21_MASK),
                                 fma(a.c_h, (double)(int)((v >> 21) & PCAL_F21_MASK),
                                     fma(a.c_l, (double)(int)(v & PCAL_F21_MASK), rr < rem ? s_q1 : s_q)));
            re = fma(S, w.x, re);
            im = fma(S, w.y, im);
            k += kstep;
            idx += istep;
            if (idx >= L) idx -= L;
        }
    } else {
#pragma unroll 1
        for (; m < m_end; m += step) {
            const double S = read_bin<false, FMT>(a, k);
            const double2 w = a.tw[idx];
            re = fma(S, w.x, re);
            im = fma(S, w.y, im);
            clear_bin<FMT>(a, k);
            k += kstep;
            idx += istep;
            if (idx >= L) idx -= L;
        }
    }
    return make_double2(re, im);
}

// Tones [i0, i1) of the N-point DFT of sP in FP32 (g threads per tone,
// combined by a fixed butterfly), written to dst[i] (shared memory of this
// CTA or, through the cluster, of another).
__device__ void dft_range(const float2* sP, const float2* sTw, int N, int i0, int i1, float2* dst) {
    const int t = threadIdx.x;
    const int ntone = i1 - i0;
    int g = 1;
    while (g < 32 && g * 2 * ntone <= (int)blockDim.x) g *= 2;
    const int groups = blockDim.x / g;
    const int gs = t % g;
#pragma unroll 1
    for (int base = 0; base < ntone; base += groups) {
        const int i = i0 + base + t / g;
        float sre = 0.f, sim = 0.f;
        if (i < i1) {
            int ix = (int)(((int64_t)i * gs) % N);
            const int step = (int)(((int64_t)i * g) % N);
#pragma unroll 4
            for (int bb = gs; bb < N; bb += g) {
                const float2 p = sP[bb];
                const float2 w = sTw[ix];
                sre = fmaf(p.x, w.x, fmaf(-p.y, w.y, sre));
                sim = fmaf(p.x, w.y, fmaf(p.y, w.x, sim));
                ix += step;
                if (ix >= N) ix -= N;
            }
        }
        for (int o = g / 2; o > 0; o >>= 1) {
            sre += __shfl_xor_sync(0xffffffffu, sre, o);
            sim += __shfl_xor_sync(0xffffffffu, sim, o);
        }
        if (i < i1 && gs == 0) dst[i] = make_float2(sre, sim);
    }
}

// The whole finalize in one cluster of C CTAs.  Thread t of every CTA takes
// residue b = t % N and every (blockDim/N)-th index m of its CTA's slice
// [per*r/C, per*(r+1)/C) of m = 0..per-1 (per = L/N), i.e. bins k = b + m*N:
// consecutive threads read consecutive bins.  Per bin: decode and rotation
// in FP64 (Eq. 3), then the bin is cleared for the next period.  The lanes of
// a residue are added in df in shared memory (fixed order).  CTA 0 then adds
// the C partials of every residue (rank order) read through distributed
// shared memory, spread over all its threads, and runs the DFT and the
// products.
// Runs in every CTA of the cluster; returns true in the CTA that wrote the
// results (rank 0), after it wrote them.
template <int FMT = -1>
__device__ __forceinline__ bool cluster_finalize(const FinArgs& a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ float4 part[kClusterThreads];  // per (lane, residue) df partials: re hi, re lo, im hi, im lo
    extern __shared__ __align__(16) uint8_t dsm[];
    const int C = (int)cluster.num_blocks(), r = (int)cluster.block_rank();
    const int N = (int)a.N;
    const ClusterSmem sm = cluster_layout(dsm, N);
    float4* Pr = sm.Pr;
    float2 *sP = sm.sP, *sTw = sm.sTw, *sT = sm.sT;
    const int t = threadIdx.x;
    // N > blockDim: one lane per residue, the residues in turns
    const bool big = N > (int)blockDim.x;
    const int lanes = big ? 1 : (int)blockDim.x / N;
    if (r == 0 || N > kClusterMaxN)
        for (int i = t; i < N; i += blockDim.x) sTw[i] = a.twN[i];
    // L <= PCAL_MAX_L: bin and rotator indices fit 32 bits (so*k does not)
    const int L = (int)a.L;
    const int per = L / N;
    const int m1 = per * (r + 1) / C;
    if (!big) {
        // thread t: residue t % N, every lanes-th m of this CTA's slice
        const int b = t % N, ml = t / N;
        if (ml < lanes) {
            const double2 z = fold_residue<FMT>(a, b, per * r / C + ml, lanes, m1);
            const df dre = df_of(z.x), dim = df_of(z.y);
            part[t] = make_float4(dre.hi, dre.lo, dim.hi, dim.lo);
        }
        __syncthreads();
        if (t < N) {
            df sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll 1
            for (int l = 0; l < lanes; ++l) {
                const float4 v = part[l * N + t];
                sr = pcal_df::add(sr, df{v.x, v.y});
                si = pcal_df::add(si, df{v.z, v.w});
            }
            Pr[t] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
        }
    } else {
        // one thread per residue, the residues in turns
#pragma unroll 1
        for (int b = t; b < N; b += blockDim.x) {
            const double2 z = fold_residue<FMT>(a, b, per * r / C, 1, m1);
            const df dre = df_of(z.x), dim = df_of(z.y);
            Pr[b] = make_float4(dre.hi, dre.lo, dim.hi, dim.lo);
        }
    }
    cluster.sync();  // every CTA's partial P is complete
    if (r == 0) {
        // residue i: the C partials in rank order, loads issued in fours;
        // G threads share a residue when N is small
        const int G = big ? 1 : (lanes < C ? lanes : C);
        const int g = big ? 0 : t / N;
        if (g < G) {
#pragma unroll 1
            for (int i = big ? t : t % N; i < N; i += big ? blockDim.x : N) {
                df sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll 1
                for (int q0 = g; q0 < C; q0 += 4 * G) {
                    float4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u * G;
                        v[u] = q < C ? *cluster.map_shared_rank(&Pr[i], q) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        sr = pcal_df::add(sr, df{v[u].x, v[u].y});
                        si = pcal_df::add(si, df{v[u].z, v[u].w});
                    }
                }
                if (big)
                    sP[i] = make_float2(sr.hi + sr.lo, si.hi + si.lo);
                else
                    part[t] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
                if (!big) break;
            }
        }
        if (!big) {
            __syncthreads();
            if (t < N) {
                df sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll 1
                for (int gg = 0; gg < G; ++gg) {
                    const float4 v = part[gg * N + t];
                    sr = pcal_df::add(sr, df{v.x, v.y});
                    si = pcal_df::add(si, df{v.z, v.w});
                }
                sP[t] = make_float2(sr.hi + sr.lo, si.hi + si.lo);
            }
        }
    }
    cluster.sync();  // P is complete in CTA 0; the other CTAs' Pr is no longer read
    if (a.Pout) {
        // the DFT runs elsewhere (the batched tensor-core DFT)
        if (r == 0)
            for (int i = t; i < N; i += blockDim.x) a.Pout[i] = sP[i];
        return false;
    }
    if (!big) {
        if (r != 0) return false;
        dft_range(sP, sTw, N, 0, N, sT);
    } else {
        // every CTA: its share of the tones from a copy of P, into CTA 0's sT
        if (r != 0) {
            const float2* p0 = cluster.map_shared_rank(sP, 0);
            for (int i = t; i < N; i += blockDim.x) sP[i] = p0[i];
        }
        __syncthreads();
        dft_range(sP, sTw, N, N * r / C, N * (r + 1) / C, cluster.map_shared_rank(sT, 0));
        cluster.sync();  // CTA 0 holds every tone; its sP is no longer read
        if (r != 0) return false;
    }
    __syncthreads();
    if (t < 32) tone_products_warp(a, sT, sm.pm.psi, sm.pm.w, sm.pm.un, sm.pm.out);
    else if (t < 64 && a.extra) peak_delay_warp(a, sP);
    __syncthreads();
    write_results_block(a, sT, sm.pm);
    return true;
}

// One instantiation per sample format: the finalize runs once per step and its
// instructions come from L2 (slow beside a streaming fold), so each plan's
// kernel holds only its own format's decode.
template <int FMT>
__global__ void __launch_bounds__(kClusterThreads, 1) fin_cluster_kernel(FinArgs a) {
    // The next fold may launch at once: it adds into the other set of bins
    // and waits for this kernel before its first atomic.
    allow_dependents();
    grid_dependency_wait();  // the bins of the preceding fold
    cluster_finalize<FMT>(a);
}

// Finalize arguments of one batched channel from its device state.
__device__ inline FinArgs batch_fin_args(const BatchChan& bc) {
    const int64_t n_tot = bc.n_abs - bc.period_start;
    FinArgs a{};
    a.fmt = bc.fmt;
    a.spilled = 1;  // 2-bit sums live in the wide arrays; the packed words are zero
    a.L = bc.L;
    a.N = bc.N;
    a.so = bc.so;
    a.q = n_tot / bc.L;
    a.rem = n_tot % bc.L;
    a.a0 = bc.period_start % bc.L;
    a.lev0 = bc.lev0;
    a.c_l = bc.c_l;
    a.c_h = bc.c_h;
    a.c_hl = bc.c_hl;
    a.M = (double)n_tot;
    a.two_over_m = n_tot > 0 ? (float)(2.0 / (double)n_tot) : 0.0f;
    a.two_pi_fc.hi = (float)bc.two_pi_fc;
    a.two_pi_fc.lo = (float)(bc.two_pi_fc - (double)a.two_pi_fc.hi);
    a.acc2 = bc.zero2;
    a.wide2 = bc.wide2;
    a.acc8 = bc.acc8;
    a.tw = bc.tw;
    a.twN = bc.twN;
    a.res = bc.res;
    a.extra = bc.res + 5 * bc.N + 3;
    a.fs_hz = bc.fs;
    return a;
}

// Batch finalize: cluster c finalizes channel c of the batch from the
// channel's device state, then starts the channel's next period.  split:
// stop after P (stored in the channel's P slot) for the batched DFT; the
// products kernel finishes the channel.  A programmatic dependent of the
// fold: it waits for the fold's bins and indices before reading any state.
__global__ void __launch_bounds__(kClusterThreads, 1) batch_fin_kernel(BatchChan* ch, const int* list, int split) {
    namespace cg = cooperative_groups;
    allow_dependents();
    grid_dependency_wait();
    const int i = (int)(blockIdx.x / cg::this_cluster().num_blocks());
    const int c = list ? list[i] : i;
    BatchChan& bc = ch[c];
    // The arguments live in shared memory: a per-thread copy passed by
    // reference to the out-of-line products went to each thread's stack, and
    // those stores (376 B x 256 threads x 16 CTAs per channel, ~88 MB for 64
    // channels) left dirty L2 lines that the next fold had to write back
    // (+50 us per C3 step).
    __shared__ FinArgs a;
    if (threadIdx.x == 0) {
        a = batch_fin_args(bc);
        if (split) a.Pout = bc.Pslot;
    }
    __syncthreads();
    // every CTA has read the state above before the first cluster barrier
    // inside, and rank 0 returns after the last one
    if (cluster_finalize(a) && threadIdx.x == 0) bc.period_start = bc.n_abs;
}

// After the batched DFT: block c runs channel c's products and
// post-processing from its tone and P slots and starts its next period.
__global__ void __launch_bounds__(kClusterThreads, 1) batch_products_kernel(BatchChan* ch) {
    BatchChan& bc = ch[blockIdx.x];
    __shared__ FinArgs a;  // in shared memory, not on every thread's stack
    if (threadIdx.x == 0) a = batch_fin_args(bc);
    __syncthreads();
    extern __shared__ __align__(16) uint8_t dsm[];
    const ClusterSmem sm = cluster_layout(dsm, bc.N);
    const int t = threadIdx.x;
    for (int i = t; i < bc.N; i += blockDim.x) {
        sm.sT[i] = bc.Tslot[i];
        sm.sP[i] = bc.Pslot[i];
    }
    __syncthreads();
    if (t < 32) tone_products_warp(a, sm.sT, sm.pm.psi, sm.pm.w, sm.pm.un, sm.pm.out);
    else if (t < 64 && a.extra) peak_delay_warp(a, sm.sP);
    __syncthreads();
    write_results_block(a, sm.sT, sm.pm);
    __syncthreads();
    if (t == 0) bc.period_start = bc.n_abs;
}

// Spread DFT for large N; the last CTA runs the products.
template <bool NoAlloc>
__global__ void fin_dft_kernel(FinArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ bool is_last;
    grid_dependency_wait();  // P of the fold kernel
    allow_dependents();
    const int64_t i0 = (int64_t)blockIdx.x * kDftTonesPerCta;
    const int64_t i1 = i0 + kDftTonesPerCta < a.N ? i0 + kDftTonesPerCta : a.N;
    float2* sP = reinterpret_cast<float2*>(smem);
    dft_tones<NoAlloc>(a, i0, i1, sP, sP + a.N, nullptr);
    __threadfence();  // the T stores of this CTA
    __syncthreads();
    if (threadIdx.x == 0) is_last = ticket_acq_rel(&a.ticket[1]) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ticket[1] = 0;
    const ProductsSmem m = products_layout(smem, a.N);
    for (int64_t i = threadIdx.x; i < a.N; i += blockDim.x) m.T[i] = __ldcg(&a.T[i]);
    __syncthreads();
    tone_products(a, m);
    if (a.extra) {
        // P again, into the shared memory the products no longer need
        __syncthreads();
        float2* sP = reinterpret_cast<float2*>(smem);
        for (int64_t b = threadIdx.x; b < a.N; b += blockDim.x) {
            const float4 v = __ldcg(&a.P[b]);
            sP[b] = make_float2(v.x + v.y, v.z + v.w);
        }
        __syncthreads();
        if (threadIdx.x < 32) peak_delay_warp(a, sP);
    }
}

__global__ void init_twiddles_kernel(double2* tw, int64_t L, float2* twN, int64_t N, int64_t sc) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < L; m += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)L, &s, &c);
        tw[m] = make_double2(c, -s);
        if (m % sc == 0 && m / sc < N) twN[m / sc] = make_float2((float)c, (float)-s);
    }
}

// Launch as a programmatic dependent of the preceding kernel in the stream.
template <typename... Args>
cudaError_t launch_pdl(void (*k)(Args...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
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
    return cudaLaunchKernelEx(&cfg, k, args...);
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

namespace {

// Launch the finalize kernels for filled-in arguments (everything but the
// work split, which is chosen here).
template <bool NoAlloc>
cudaError_t launch_finalize_args(FinArgs a, int num_sms, cudaStream_t s, int* launches) {
    const int64_t N = a.N;
    int G = (int)(N < num_sms ? N : num_sms);
    a.bc = (int)((N + G - 1) / G);
    G = (int)((N + a.bc - 1) / a.bc);
    // tpb = the largest power of two with bc*tpb <= 256; the block is a
    // multiple of 32 threads (the shuffles and the DFT need whole warps)
    a.tpb = 1;
    while (a.bc * a.tpb * 2 <= 256) a.tpb *= 2;
    const int threads = (a.bc * a.tpb + 31) / 32 * 32;
    size_t smem = (size_t)threads * 16;
    if (N <= kDftInFoldMaxN) {
        const size_t need = products_bytes(N) + (size_t)N * 16;  // products + P + twiddles
        if (need > smem) smem = need;
    }
    cudaError_t e = cudaSuccess;
    static size_t fold_smem_set = 0;
    if (smem > 48 * 1024 && smem > fold_smem_set) {
        e = cudaFuncSetAttribute(fin_fold_kernel<NoAlloc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fold_smem_set = smem;
    }
    e = launch_pdl(fin_fold_kernel<NoAlloc>, G, threads, smem, s, a);
    *launches += 1;
    if (e != cudaSuccess || N <= kDftInFoldMaxN) return e;
    const int threads2 = 256;
    const size_t smem2 = (size_t)N * 16 > products_bytes(N) ? (size_t)N * 16 : products_bytes(N);
    static size_t dft_smem_set = 0;
    if (smem2 > 48 * 1024 && smem2 > dft_smem_set) {
        e = cudaFuncSetAttribute(fin_dft_kernel<NoAlloc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        if (e != cudaSuccess) return e;
        dft_smem_set = smem2;
    }
    e = launch_pdl(fin_dft_kernel<NoAlloc>, (int)((N + kDftTonesPerCta - 1) / kDftTonesPerCta), threads2, smem2, s, a);
    *launches += 1;
    return e;
}

// Cluster size for fin_cluster_kernel on the current device: 16 CTAs where
// the device can co-schedule them (a non-portable size), else the portable
// 8; 0 when no cluster fits.  Evaluated once per device.
int cluster_size_for_device() {
    static std::mutex mu;
    static int cached[64];
    static bool known[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (known[dev]) return cached[dev];
    int best = 0;
    for (auto k : {fin_cluster_kernel<PCAL_2BIT>, fin_cluster_kernel<PCAL_I8>, fin_cluster_kernel<PCAL_F32>})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            (void)cudaGetLastError();
    for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kClusterThreads);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, fin_cluster_kernel<PCAL_2BIT>, &cfg) == cudaSuccess && n > 0) {
            best = c;
            break;
        }
        (void)cudaGetLastError();
    }
    cached[dev] = best;
    known[dev] = true;
    return best;
}

// One cluster of C CTAs as a programmatic dependent of the preceding kernel.
// The CTAs ask for kClusterPadSmem more shared memory than they use, so that
// none of them fits on an SM beside a CTA of the fold that overlaps it (about
// 205 KB each): sharing an SM with a fold CTA slowed the finalize 2-3x.  The
// fold leaves kFinalizeReserveSms SMs for it.
cudaError_t launch_cluster_finalize(const FinArgs& a, int C, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = cluster_smem_bytes(a.N) + kClusterPadSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = C;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    if (a.fmt == PCAL_2BIT) return cudaLaunchKernelEx(&cfg, fin_cluster_kernel<PCAL_2BIT>, a);
    if (a.fmt == PCAL_I8) return cudaLaunchKernelEx(&cfg, fin_cluster_kernel<PCAL_I8>, a);
    return cudaLaunchKernelEx(&cfg, fin_cluster_kernel<PCAL_F32>, a);
}

// Finalize of a long-period plan (one CTA): the lanes of each bin added in
// df (lane order), then the DFT, the products and the post-processing of the
// folded path.
__global__ void __launch_bounds__(kClusterThreads) rot_finalize_kernel(FinArgs a, const float4* acc, int lanes) {
    __shared__ float4 part[kClusterThreads];
    extern __shared__ __align__(16) uint8_t dsm[];
    const int N = (int)a.N;
    const ClusterSmem sm = cluster_layout(dsm, N);
    const int t = threadIdx.x;
    for (int i = t; i < N; i += blockDim.x) sm.sTw[i] = a.twN[i];
    // bin b: its lanes split over G threads, then the G partials in order
    const int G = (int)blockDim.x / N > 0 ? (int)blockDim.x / N : 1;
    const int per_round = (int)blockDim.x / G;
    for (int b0 = 0; b0 < N; b0 += per_round) {
        const int b = b0 + t / G, g = t % G;
        df sr{0.f, 0.f}, si{0.f, 0.f};
        if (t / G < per_round && b < N)
            for (int l = g; l < lanes; l += G) {
                const float4 v = acc[(int64_t)l * N + b];
                sr = pcal_df::add(sr, df{v.x, v.y});
                si = pcal_df::add(si, df{v.z, v.w});
            }
        part[t] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
        __syncthreads();
        if (g == 0 && t / G < per_round && b < N) {
            df tr{0.f, 0.f}, ti{0.f, 0.f};
            for (int q = 0; q < G; ++q) {
                const float4 v = part[t + q];
                tr = pcal_df::add(tr, df{v.x, v.y});
                ti = pcal_df::add(ti, df{v.z, v.w});
            }
            sm.sP[b] = make_float2(tr.hi + tr.lo, ti.hi + ti.lo);
        }
        __syncthreads();
    }
    dft_range(sm.sP, sm.sTw, N, 0, N, sm.sT);
    __syncthreads();
    if (t < 32) tone_products_warp(a, sm.sT, sm.pm.psi, sm.pm.w, sm.pm.un, sm.pm.out);
    else if (t < 64) peak_delay_warp(a, sm.sP);
    __syncthreads();
    write_results_block(a, sm.sT, sm.pm);
}

}  // namespace

cudaError_t launch_rot_finalize(const float4* acc, int lanes, int N, double fs, double fc, int64_t M,
                                const float2* twN, double* res, cudaStream_t s) {
    FinArgs a{};
    a.N = N;
    a.L = N;
    a.fs_hz = fs;
    a.M = (double)M;
    a.two_over_m = M > 0 ? (float)(2.0 / (double)M) : 0.0f;
    const double tpf = 6.283185307179586476925 * fc;
    a.two_pi_fc.hi = (float)tpf;
    a.two_pi_fc.lo = (float)(tpf - (double)a.two_pi_fc.hi);
    a.twN = twN;
    a.res = res;
    a.extra = res + 5 * (int64_t)N + 3;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(rot_finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)cluster_smem_bytes(kClusterBigN));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    rot_finalize_kernel<<<1, kClusterThreads, cluster_smem_bytes(N), s>>>(a, acc, lanes);
    return cudaGetLastError();
}

cudaError_t prepare_batch_finalize() {
    const int C = cluster_size_for_device();
    if (C == 0) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(batch_fin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cluster_smem_bytes(kClusterBigN));
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(batch_fin_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_products_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cluster_smem_bytes(kClusterBigN));
    return e;
}

cudaError_t launch_batch_products(BatchChan* d_ch, int n_ch, int max_n, cudaStream_t s) {
    if (max_n > kClusterBigN) return cudaErrorInvalidValue;
    batch_products_kernel<<<n_ch, kClusterThreads, cluster_smem_bytes(max_n), s>>>(d_ch);
    return cudaGetLastError();
}

// prepare_batch_finalize() must have succeeded on this device (it makes the
// CUDA calls that a stream capture does not allow).  max_n: the largest N of
// the batch's channels.
cudaError_t launch_batch_finalize(BatchChan* d_ch, int n_ch, int max_n, const int* d_list, cudaStream_t s, int split) {
    // 8-CTA clusters: with one cluster per channel the launch is several waves
    // of CTAs, and fewer, longer clusters finish sooner (64 channels of up to
    // L 25600: 16 CTAs 53 us, 8 CTAs 43 us, 4 CTAs 57 us; same phasors)
    int C = cluster_size_for_device();
    if (C > 8) C = 8;
    if (C == 0) return cudaErrorNotSupported;
    if (max_n > kClusterBigN) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_ch * C);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = cluster_smem_bytes(max_n);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, batch_fin_kernel, d_ch, d_list, split);
}

namespace {

void set_common(FinArgs& a, const pcal_geometry& g, int64_t n_tot) {
    a.fs_hz = (double)g.fs;
    a.L = g.L;
    a.N = g.N;
    a.so = g.step_offset;
    a.M = (double)n_tot;
    a.two_over_m = n_tot > 0 ? (float)(2.0 / (double)n_tot) : 0.0f;
    const double tpf = 6.283185307179586476925 * (double)g.f_comb;
    a.two_pi_fc.hi = (float)tpf;
    a.two_pi_fc.lo = (float)(tpf - (double)a.two_pi_fc.hi);
}

}  // namespace

cudaError_t launch_finalize(pcal_plan* p, cudaStream_t s) {
    FinArgs a{};
    const pcal_geometry& g = p->g;
    const int64_t n_tot = p->n_abs - p->period_start;
    set_common(a, g, n_tot);
    a.fmt = g.format;
    a.spilled = p->spilled ? 1 : 0;
    a.q = n_tot / g.L;
    a.rem = n_tot % g.L;
    a.a0 = p->period_start % g.L;
    const double* lv = p->levels;
    a.lev0 = lv[0];
    a.c_l = lv[1] - lv[0];
    a.c_h = lv[2] - lv[0];
    a.c_hl = lv[3] - lv[2] - lv[1] + lv[0];
    a.acc2 = cur_acc2(p);
    a.wide2 = cur_wide2(p);
    a.acc8 = cur_acc8(p);
    a.accf = cur_accf(p);
    if (g.format == PCAL_F32) {
        for (int e = 0; e < p->n_pending; ++e) {
            a.pf[e] = p->pending[e].base;
            a.pf_rg[e] = p->pending[e].row_groups;
            a.pf_ka[e] = p->pending[e].k_a;
        }
        a.n_pf = p->n_pending;
        a.pf_cols = g.row_samples / g.samples_per_byte_x4;
    }
    a.tw = p->d_tw;
    a.twN = p->d_twN;
    a.P = reinterpret_cast<float4*>(p->d_P);
    a.T = reinterpret_cast<float2*>(p->d_T);
    a.res = p->d_res;
    a.extra = p->d_res + 5 * g.N + 3;
    a.ticket = p->d_ticket;
    cudaError_t e = cudaErrorUnknown;
    bool done = false;
    if (g.N <= kClusterMaxN && g.L <= kClusterMaxL) {
        const int C = cluster_size_for_device();
        if (C > 0) {
            p->stats.kernel_launches += 1;
            e = launch_cluster_finalize(a, C, s);
            done = true;
        }
    }
    if (!done) {
        int launches = 0;
        e = launch_finalize_args<false>(a, p->num_sms, s, &launches);
        p->stats.kernel_launches += launches;
    }
    if (e == cudaSuccess) p->n_pending = 0;  // the finalize added them (and clears the bins)
    return e;
}

// ---- finalize without any allocation -------------------------------------------
//
// Some callers cannot allocate GPU memory at all: code running inside a
// pre-sized memory pool or arena, a process whose device memory budget is
// fixed at start-up, or a stream that is being captured into a CUDA graph,
// where a cudaMalloc is not allowed.  For them pcal_tones_from_counts_noalloc
// runs the finalize kernels with their scratch (the folded bins P, the tone
// phasors T and the completion tickets) in the file-scope array below, which
// every GPU that loads this library holds until the process exits; the
// rotator and DFT twiddles are evaluated on the fly instead of read from a
// plan's tables.  Everything else comes from the caller.

namespace {

constexpr int kNoAllocMaxN = 1024;

struct NoAllocScratch {
    float4 P[kNoAllocMaxN];
    float2 T[kNoAllocMaxN];
    unsigned int ticket[4];
};

// ~24.6 KB per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoAllocScratch* g_noalloc_ptr[kMaxDevices];  // device address of the array, per device
int g_noalloc_sms[kMaxDevices];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
cudaError_t noalloc_scratch(NoAllocScratch** out, int* num_sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&g_noalloc_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<NoAllocScratch*>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    *num_sms = g_noalloc_sms[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int pcal_tones_from_counts_noalloc(double fs, double f_comb, double f_offset, int N,
                                              const int64_t* d_counts, int64_t n_samples, const double levels[4],
                                              double* d_results, void* stream) {
    pcal_geometry g;
    int rc = pcal_plan_geometry(fs, f_comb, f_offset, N, PCAL_2BIT, &g);
    if (rc != PCAL_OK) return rc;
    if (g.N > kNoAllocMaxN) return PCAL_ETOOLARGE;
    if (!d_counts || !d_results || !levels || n_samples < 0) return PCAL_EINVAL;
    for (int i = 0; i < 4; ++i)
        if (!(levels[i] == levels[i]) || levels[i] > 1e300 || levels[i] < -1e300) return PCAL_EINVAL;
    NoAllocScratch* sc = nullptr;
    int num_sms = 0;
    cudaError_t e = noalloc_scratch(&sc, &num_sms);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PCAL_ENOMEM : PCAL_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the completion tickets must start at zero (the array keeps whatever the
    // previous call, possibly an interrupted one, left there)
    e = cudaMemsetAsync(sc->ticket, 0, sizeof(sc->ticket), s);
    if (e != cudaSuccess) return PCAL_ECUDA;
    FinArgs a{};
    set_common(a, g, n_samples);
    a.fmt = PCAL_2BIT;
    a.counts4 = reinterpret_cast<const long long*>(d_counts);
    for (int i = 0; i < 4; ++i) a.lev[i] = levels[i];
    a.tw = nullptr;   // rotator evaluated per bin (no plan table)
    a.twN = nullptr;  // DFT twiddles evaluated per CTA
    a.P = sc->P;
    a.T = sc->T;
    a.ticket = sc->ticket;
    a.res = d_results;
    int launches = 0;
    e = launch_finalize_args<true>(a, num_sms, s, &launches);
    return e == cudaSuccess ? PCAL_OK : PCAL_ECUDA;
}
