/*
 * FP64 CPU ORACLE for multi-tone phase-calibration extraction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code with the CUDA path and must never be used to produce a product
 * result.
 *
 * What it computes (paper Sec. 2):
 *   Eq. 1   x[n] = s[n] + sum_i sin((i*w_comb + w_offset)*n + phi_i)
 *   Eq. 3   xhat[n] = x[n] * exp(-j*w_offset*n)          (rotation)
 *   Eq. 2   P[b] = sum_j xhat[b + j*N_bins]                (time-domain fold)
 *   DFT(P)  T_i = sum_b P[b] exp(-j*2*pi*i*b/N_bins)       (tone phasors)
 * Together these equal the direct definition used by `orc_direct`:
 *   T_i = sum_n x[n] * exp(-j*theta_i*n),  theta_i = 2*pi*(i*fc + fo)/fs,
 * with n the absolute sample index.  The phase argument is reduced exactly in
 * integers: with g = gcd(fs, fc, fo) and L = fs/g (Eq. 4 combined with the
 * N_bins period), theta_i*n = 2*pi*(((i*fc + fo)/g * n) mod L)/L, so a table of
 * the L values exp(-j*2*pi*m/L), evaluated with the C library's cos/sin in
 * FP64, serves every tone.  All sums use Neumaier compensation.
 *
 * Readings (where the paper is silent or its listings disagree): the rotation
 * sign is exp(-j...) as in Eq. 3 (the listings use +sin); the DFT is the
 * forward exp(-j...) transform with no normalisation; 2-bit codes are
 * (h<<1)|l, four per byte, least significant sample first, decoded through a
 * 4-entry level table.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Planted-mistake switch for the oracle's own self-tests (0 = none). */
static int g_mutation = 0;
void orc_set_mutation(int m) { g_mutation = m; }
int orc_get_mutation(void) { return g_mutation; }

/* 1: rotation sign flipped (exp(+j..)); 2: tone index off by one; 3: absolute
 * phase reference dropped (n0 ignored); 4: 2-bit h/l bits swapped; 5: fold
 * period off by one (L-1); 6: rotator indexed by the folded bin (rotate after
 * folding instead of before). */
enum { MUT_NONE = 0, MUT_ROT_SIGN = 1, MUT_TONE_INDEX = 2, MUT_DROP_N0 = 3, MUT_SWAP_HL = 4, MUT_FOLD_PERIOD = 5,
       MUT_ROTATE_AFTER_FOLD = 6 };

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a < 0 ? -a : a;
}

/* Eq. 4 and the N_bins period: returns 0 and fills N, L, the integer tone
 * step of the comb (fc/g) and of the offset (fo/g), or -1 if the plan is not
 * representable with integral frequencies. */
int orc_plan(int64_t fs, int64_t fc, int64_t fo, int64_t* N, int64_t* L, int64_t* sc, int64_t* so) {
    if (fs <= 0 || fc <= 0 || fo < 0 || fs % fc != 0) return -1;
    int64_t g = gcd64(gcd64(fs, fc), fo);
    *N = fs / fc;
    *L = fs / g;
    *sc = fc / g;
    *so = fo / g;
    return 0;
}

/* exp(-j*2*pi*m/L) for m = 0..L-1, interleaved re/im. */
static double* twiddles(int64_t L) {
    double* tw = (double*)malloc((size_t)L * 2 * sizeof(double));
    if (!tw) return NULL;
    double s = (g_mutation == MUT_ROT_SIGN) ? 1.0 : -1.0;
    for (int64_t m = 0; m < L; ++m) {
        double a = 6.283185307179586476925 * (double)m / (double)L;
        tw[2 * m] = cos(a);
        tw[2 * m + 1] = s * sin(a);
    }
    return tw;
}

typedef struct {
    double s, c;
} nsum; /* Neumaier compensated sum */

static inline void nadd(nsum* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum* a) { return a->s + a->c; }

/* Sample t of a stream: fmt 0 = float32, 1 = int8, 2 = 2-bit packed codes,
 * 3 = float64 (used by the oracle's own exact self-tests). */
static inline int code_of(const uint8_t* b, int64_t t) {
    int c = (b[t >> 2] >> (2 * (int)(t & 3))) & 3;
    if (g_mutation == MUT_SWAP_HL) c = ((c & 1) << 1) | (c >> 1);
    return c;
}
static inline double sample_at(const void* buf, int fmt, int64_t t, const double* lev) {
    if (fmt == 0) return (double)((const float*)buf)[t];
    if (fmt == 1) return (double)((const int8_t*)buf)[t];
    if (fmt == 3) return ((const double*)buf)[t];
    return lev[code_of((const uint8_t*)buf, t)];
}

/*
 * Direct definition, O(M*N):  T_i = sum_{t<M} x[t] exp(-j*theta_i*(n0+t)),
 * i = 0..n_tones-1.  out holds n_tones complex values, interleaved re/im.
 */
int orc_direct(const void* buf, int fmt, const double* levels, int64_t M, int64_t n0, int64_t fs, int64_t fc,
               int64_t fo, int64_t n_tones, double* out) {
    int64_t N, L, sc, so;
    if (M < 0 || n0 < 0 || orc_plan(fs, fc, fo, &N, &L, &sc, &so) != 0) return -1;
    double* tw = twiddles(L);
    if (!tw) return -2;
    if (g_mutation == MUT_DROP_N0) n0 = 0;
    for (int64_t i = 0; i < n_tones; ++i) {
        int64_t ii = (g_mutation == MUT_TONE_INDEX) ? i + 1 : i;
        int64_t a = (ii * sc + so) % L; /* tone step in units of 2*pi/L */
        nsum re = {0, 0}, im = {0, 0};
        int64_t k = n0 % L;          /* (n0 + t) mod L          */
        int64_t r = (a * k) % L;     /* (a * (n0 + t)) mod L     */
        for (int64_t t = 0; t < M; ++t) {
            double x = sample_at(buf, fmt, t, levels);
            nadd(&re, x * tw[2 * r]);
            nadd(&im, x * tw[2 * r + 1]);
            if (++k == L) {
                k = 0;
                r = 0;
            } else {
                r += a;
                if (r >= L) r -= L;
            }
        }
        out[2 * i] = nval(&re);
        out[2 * i + 1] = nval(&im);
    }
    free(tw);
    return 0;
}

/*
 * Direct definition for any offset that is a binary fraction of a hertz,
 * f_offset = fo_num / 2^fo_shift (prime offsets whose period L is too long to
 * fold, and non-integral offsets):
 *   T_i = sum_t x[t] exp(-j*2*pi*((i*fc*2^s + fo_num)*(n0+t) mod (fs*2^s)) / (fs*2^s)),
 * the phase reduced exactly in 128-bit integers, cos/sin per term, Neumaier sums.
 */
int orc_direct_dy(const void* buf, int fmt, const double* levels, int64_t M, int64_t n0, int64_t fs, int64_t fc,
                  int64_t fo_num, int fo_shift, int64_t n_tones, double* out) {
    typedef __int128 i128;
    if (M < 0 || n0 < 0 || fs <= 0 || fc <= 0 || fo_num < 0 || fo_shift < 0 || fo_shift > 60) return -1;
    if (g_mutation == MUT_DROP_N0) n0 = 0;
    const i128 mod = (i128)fs << fo_shift;
    const double sgn = (g_mutation == MUT_ROT_SIGN) ? 1.0 : -1.0;
    for (int64_t i = 0; i < n_tones; ++i) {
        int64_t ii = (g_mutation == MUT_TONE_INDEX) ? i + 1 : i;
        const i128 a = ((((i128)ii * fc) << fo_shift) + fo_num) % mod;
        i128 r = (a * (i128)n0) % mod;
        nsum re = {0, 0}, im = {0, 0};
        for (int64_t t = 0; t < M; ++t) {
            const double x = sample_at(buf, fmt, t, levels);
            const double ang = 6.283185307179586476925 * ((double)r / (double)mod);
            nadd(&re, x * cos(ang));
            nadd(&im, x * sgn * sin(ang));
            r += a;
            if (r >= mod) r -= mod;
        }
        out[2 * i] = nval(&re);
        out[2 * i + 1] = nval(&im);
    }
    return 0;
}

/*
 * Fold of the raw stream modulo L (Eq. 2 with the combined period):
 * S[k] = sum_{t : (n0+t) mod L == k} x[t], FP64 with compensation.
 */
int orc_fold_real(const void* buf, int fmt, const double* levels, int64_t M, int64_t n0, int64_t L, double* S) {
    if (M < 0 || n0 < 0 || L <= 0) return -1;
    nsum* acc = (nsum*)calloc((size_t)L, sizeof(nsum));
    if (!acc) return -2;
    if (g_mutation == MUT_DROP_N0) n0 = 0;
    int64_t per = (g_mutation == MUT_FOLD_PERIOD && L > 1) ? L - 1 : L;
    int64_t k = n0 % per;
    for (int64_t t = 0; t < M; ++t) {
        nadd(&acc[k], sample_at(buf, fmt, t, levels));
        if (++k == per) k = 0;
    }
    for (int64_t j = 0; j < L; ++j) S[j] = nval(&acc[j]);
    free(acc);
    return 0;
}

/*
 * Tone phasors from L folded real bins by the direct bin sum:
 * T_i = sum_{k<L} S[k] exp(-j*theta_i*k).  Identical to orc_direct because
 * theta_i*L is a multiple of 2*pi.
 */
int orc_tones_from_bins(const double* S, int64_t fs, int64_t fc, int64_t fo, int64_t n_tones, double* out) {
    int64_t N, L, sc, so;
    if (orc_plan(fs, fc, fo, &N, &L, &sc, &so) != 0) return -1;
    double* tw = twiddles(L);
    if (!tw) return -2;
    for (int64_t i = 0; i < n_tones; ++i) {
        int64_t ii = (g_mutation == MUT_TONE_INDEX) ? i + 1 : i;
        int64_t a = (ii * sc + so) % L;
        nsum re = {0, 0}, im = {0, 0};
        int64_t r = 0;
        for (int64_t k = 0; k < L; ++k) {
            nadd(&re, S[k] * tw[2 * r]);
            nadd(&im, S[k] * tw[2 * r + 1]);
            r += a;
            if (r >= L) r -= L;
        }
        out[2 * i] = nval(&re);
        out[2 * i + 1] = nval(&im);
    }
    free(tw);
    return 0;
}

/*
 * The paper's own route from L real bins to N tone phasors:
 *   rotate each bin by exp(-j*w_offset*k)       (Eq. 3; the rotator repeats
 *                                                 with the period of Eq. 4),
 *   fold the L rotated bins to N_bins = fs/fc    (Eq. 2),
 *   N_bins-point forward DFT                     (DFT(P), Sec. 2).
 * Twiddles of the N_bins-point DFT are entries of the same L-point table,
 * since L/N_bins = fc/g is an integer.
 */
int orc_rotate_fold_dft(const double* S, int64_t fs, int64_t fc, int64_t fo, double* out /* 2*N */) {
    int64_t N, L, sc, so;
    if (orc_plan(fs, fc, fo, &N, &L, &sc, &so) != 0) return -1;
    double* tw = twiddles(L);
    if (!tw) return -2;
    nsum* P = (nsum*)calloc((size_t)N * 2, sizeof(nsum));
    if (!P) {
        free(tw);
        return -2;
    }
    for (int64_t k = 0; k < L; ++k) {
        int64_t b = k % N;
        int64_t kr = (g_mutation == MUT_ROTATE_AFTER_FOLD) ? b : k;
        int64_t r = (so * kr) % L;                  /* rotator phase index */
        nadd(&P[2 * b], S[k] * tw[2 * r]);
        nadd(&P[2 * b + 1], S[k] * tw[2 * r + 1]);
    }
    for (int64_t i = 0; i < N; ++i) {
        nsum re = {0, 0}, im = {0, 0};
        for (int64_t b = 0; b < N; ++b) {
            int64_t m = ((i * b) % N) * sc;           /* exp(-j*2*pi*i*b/N)  */
            double pr = nval(&P[2 * b]), pi = nval(&P[2 * b + 1]);
            double wr = tw[2 * m], wi = tw[2 * m + 1];
            nadd(&re, pr * wr - pi * wi);
            nadd(&im, pr * wi + pi * wr);
        }
        out[2 * i] = nval(&re);
        out[2 * i + 1] = nval(&im);
    }
    free(P);
    free(tw);
    return 0;
}

/*
 * Exact per-(bin, code) counts of a 2-bit stream:
 * counts[4*k + c] = #{t < M : (n0+t) mod L == k and code(t) == c}.
 */
int orc_counts_2bit(const uint8_t* bytes, int64_t M, int64_t n0, int64_t L, int64_t* counts) {
    if (M < 0 || n0 < 0 || L <= 0) return -1;
    memset(counts, 0, (size_t)L * 4 * sizeof(int64_t));
    if (g_mutation == MUT_DROP_N0) n0 = 0;
    int64_t per = (g_mutation == MUT_FOLD_PERIOD && L > 1) ? L - 1 : L;
    int64_t k = n0 % per;
    for (int64_t t = 0; t < M; ++t) {
        counts[4 * k + code_of(bytes, t)] += 1;
        if (++k == per) k = 0;
    }
    return 0;
}

/* Exact per-bin sums of an int8 stream: S[k] = sum_{(n0+t) mod L == k} x[t]. */
int orc_sums_i8(const int8_t* x, int64_t M, int64_t n0, int64_t L, int64_t* S) {
    if (M < 0 || n0 < 0 || L <= 0) return -1;
    memset(S, 0, (size_t)L * sizeof(int64_t));
    if (g_mutation == MUT_DROP_N0) n0 = 0;
    int64_t per = (g_mutation == MUT_FOLD_PERIOD && L > 1) ? L - 1 : L;
    int64_t k = n0 % per;
    for (int64_t t = 0; t < M; ++t) {
        S[k] += x[t];
        if (++k == per) k = 0;
    }
    return 0;
}

/* Real bins from 2-bit counts: S[k] = sum_c levels[c] * counts[4k + c]. */
int orc_decode_counts(const int64_t* counts, int64_t L, const double* levels, double* S) {
    for (int64_t k = 0; k < L; ++k) {
        nsum a = {0, 0};
        for (int c = 0; c < 4; ++c) nadd(&a, levels[c] * (double)counts[4 * k + c]);
        S[k] = nval(&a);
    }
    return 0;
}
