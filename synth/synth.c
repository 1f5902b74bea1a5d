/*
 * Seeded synthetic baseband streams for multi-tone phase-calibration tests.
 *
 * This module only MAKES inputs. It holds none of the extraction method's
 * arithmetic (no rotation, no folding, no DFT) and is shared by the CPU oracle
 * tests and by the GPU benchmarks, so that both sides consume identical bytes.
 *
 * Signal model (paper Sec. 2, Eq. 1):
 *     x[n] = sigma * z[n] + sum_{i=0}^{N-1} A * sin(2*pi*(i*fc + fo)*(n/fs + td))
 * with z[n] ~ N(0,1).  The tone phase phi_i = (i*w_comb + w_offset)*td*fs of
 * Eq. 1 is 2*pi*(i*fc + fo)*td.  n is the ABSOLUTE sample index of the stream.
 * The comb term is periodic in n with period L = fs / gcd(fs, fc, fo), so it
 * is tabulated once per call over one period, with its phase argument reduced
 * exactly in integers: ((i*fc + fo) * k) mod fs.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from its published
 * definition, keyed by the 64-bit seed; the counter is (pair index lo, pair
 * index hi, stream id, 0).  Each counter value gives two 53-bit uniforms and,
 * through the Box-Muller transform, the normals z[2m] and z[2m+1].
 *
 * Quantisers (readings: Sec. 1 fixes only a sample width of 2 bits or more):
 *   f32 : float32(x)
 *   i8  : clamp(round-half-even(scale * x), -128, 127)
 *   2bit: code 0: x < -t, 1: -t <= x < 0, 2: 0 <= x < t, 3: x >= t
 *         (bit1 = sign bit h, bit0 = magnitude-sign bit l), four samples per
 *         byte, sample j of a byte in bits 2j..2j+1 (least significant first).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t o0 = hi1 ^ c[1] ^ k[0];
    uint32_t o2 = hi0 ^ c[3] ^ k[1];
    c[0] = o0;
    c[1] = lo1;
    c[2] = o2;
    c[3] = lo0;
}

/* Philox4x32 with R rounds; the key is bumped between rounds. */
void synth_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], int rounds, uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < rounds; ++r) {
        if (r > 0) {
            k[0] += PHILOX_W0;
            k[1] += PHILOX_W1;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

static inline double u53(uint32_t a, uint32_t b) {
    /* (0,1): 27 high bits of a, 26 high bits of b, offset by half a step. */
    uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

/* Two standard normals for pair index m of stream `stream`. */
static inline void normal_pair(uint64_t seed, uint32_t stream, uint64_t m, double* z0, double* z1) {
    uint32_t ctr[4] = {(uint32_t)m, (uint32_t)(m >> 32), stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    synth_philox4x32(ctr, key, 10, o);
    double u1 = u53(o[0], o[1]);
    double u2 = u53(o[2], o[3]);
    double r = sqrt(-2.0 * log(u1));
    double a = 6.283185307179586476925 * u2;
    *z0 = r * cos(a);
    *z1 = r * sin(a);
}

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a < 0 ? -a : a;
}

/* One period of the comb of Eq. 1; returns its length L, or -1 on bad input. */
static int64_t comb_table(int64_t fs, int64_t fc, int64_t fo, int64_t N, double A, double td, double** out) {
    if (fs <= 0 || fc <= 0 || fo < 0 || N < 0) return -1;
    int64_t L = fs / gcd64(gcd64(fs, fc), fo);
    double* p = (double*)calloc((size_t)L, sizeof(double));
    if (!p) return -1;
    if (A != 0.0) {
        for (int64_t i = 0; i < N; ++i) {
            int64_t f = i * fc + fo;              /* tone frequency in Hz      */
            int64_t step = f % fs;                /* phase step, units of 1/fs */
            double phi = 6.283185307179586476925 * fmod((double)f * td, 1.0);
            int64_t r = 0;                         /* (step * k) mod fs, exact  */
            for (int64_t k = 0; k < L; ++k) {
                p[k] += A * sin(6.283185307179586476925 * ((double)r / (double)fs) + phi);
                r += step;
                if (r >= fs) r -= fs;
            }
        }
    }
    *out = p;
    return L;
}

/*
 * Offsets that are not whole hertz, or whose period L is too long to tabulate:
 * f_offset = fo_num / 2^fo_shift exactly (every binary fraction is such a
 * ratio), tone i at f_i = (i*fc*2^s + fo_num) / 2^s.  Its phase at sample n
 * is 2*pi*((i*fc*2^s + fo_num)*n mod (fs*2^s)) / (fs*2^s) + 2*pi*f_i*td,
 * reduced exactly in 128-bit integers; the comb is summed tone by tone.
 * Returns the comb values for n0 .. n0+count-1 into p (count doubles).
 */
typedef __int128 i128;
static int comb_direct(int64_t fs, int64_t fc, int64_t fo_num, int fo_shift, int64_t N, double A, double td,
                       int64_t n0, int64_t count, double* p) {
    if (fs <= 0 || fc <= 0 || fo_num < 0 || fo_shift < 0 || fo_shift > 60 || N < 0) return -1;
    for (int64_t t = 0; t < count; ++t) p[t] = 0.0;
    if (A == 0.0) return 0;
    const i128 mod = (i128)fs << fo_shift;
    for (int64_t i = 0; i < N; ++i) {
        const i128 a = (((i128)i * fc) << fo_shift) + fo_num; /* f_i * 2^s                 */
        const double fi = (double)a / ldexp(1.0, fo_shift);
        const double phi = 6.283185307179586476925 * fmod(fi * td, 1.0);
        const i128 step = a % mod;
        i128 r = (step * (i128)n0) % mod;                     /* (a*n) mod (fs*2^s), exact */
        for (int64_t t = 0; t < count; ++t) {
            p[t] += A * sin(6.283185307179586476925 * ((double)r / (double)mod) + phi);
            r += step;
            if (r >= mod) r -= mod;
        }
    }
    return 0;
}

/*
 * Real samples x[n] for absolute indices n0 .. n0+count-1, written as FP64.
 * The noise of absolute index n comes from pair m = n/2 (even n: first normal).
 */
int synth_real(uint64_t seed, uint32_t stream, int64_t n0, int64_t count, double sigma, int64_t fs, int64_t fc,
               int64_t fo, int64_t N, double A, double td, double* out) {
    if (n0 < 0 || count < 0) return -1;
    double* p = NULL;
    int64_t L = comb_table(fs, fc, fo, N, A, td, &p);
    if (L <= 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < (count + 4095) / 4096; ++blk) {
        int64_t s = blk * 4096, e = s + 4096 < count ? s + 4096 : count;
        int64_t k = (n0 + s) % L;
        for (int64_t t = s; t < e; ++t) {
            int64_t n = n0 + t;
            double z = 0.0;
            if (sigma != 0.0) {
                double z0, z1;
                normal_pair(seed, stream, (uint64_t)n >> 1, &z0, &z1);
                z = (n & 1) ? z1 : z0;
            }
            out[t] = sigma * z + p[k];
            if (++k == L) k = 0;
        }
    }
    free(p);
    return 0;
}

static inline uint8_t code2(double x, double t) {
    /* h = sign bit, l = magnitude bit XOR'd so that codes are monotone in x. */
    if (x >= 0.0) return x >= t ? 3u : 2u;
    return x >= -t ? 1u : 0u;
}

static inline int8_t quant8(double x, double scale) {
    double y = nearbyint(scale * x); /* default rounding mode: half to even */
    if (y > 127.0) y = 127.0;
    if (y < -128.0) y = -128.0;
    return (int8_t)y;
}

/*
 * Quantised streams.  fmt 0: float32, 1: int8 (param = scale), 2: 2-bit packed
 * (param = threshold t in units of sigma=1 signal; count must be a multiple of 4).
 * Works block by block so that very long streams need no FP64 copy.
 */
int synth_quantized(uint64_t seed, uint32_t stream, int64_t n0, int64_t count, double sigma, int64_t fs, int64_t fc,
                    int64_t fo, int64_t N, double A, double td, int fmt, double param, void* out) {
    if (n0 < 0 || count < 0) return -1;
    if (fmt == 2 && (count % 4) != 0) return -1;
    double* p = NULL;
    int64_t L = comb_table(fs, fc, fo, N, A, td, &p);
    if (L <= 0) return -1;
    int64_t nblk = (count + 65535) / 65536;
    int err = 0;
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nblk; ++blk) {
        int64_t s = blk * 65536, e = s + 65536 < count ? s + 65536 : count;
        int64_t k = (n0 + s) % L;
        uint8_t acc = 0;
        for (int64_t t = s; t < e; ++t) {
            int64_t n = n0 + t;
            double z = 0.0;
            if (sigma != 0.0) {
                double z0, z1;
                normal_pair(seed, stream, (uint64_t)n >> 1, &z0, &z1);
                z = (n & 1) ? z1 : z0;
            }
            double x = sigma * z + p[k];
            if (++k == L) k = 0;
            if (fmt == 0) {
                ((float*)out)[t] = (float)x;
            } else if (fmt == 1) {
                ((int8_t*)out)[t] = quant8(x, param);
            } else {
                acc |= (uint8_t)(code2(x, param) << (2 * (t & 3)));
                if ((t & 3) == 3) {
                    ((uint8_t*)out)[t >> 2] = acc;
                    acc = 0;
                }
            }
        }
    }
    (void)err;
    free(p);
    return 0;
}

/*
 * As synth_real / synth_quantized for an offset fo_num / 2^fo_shift Hz (see
 * comb_direct): the comb is evaluated sample by sample, in blocks.
 */
int synth_real_dy(uint64_t seed, uint32_t stream, int64_t n0, int64_t count, double sigma, int64_t fs, int64_t fc,
                  int64_t fo_num, int fo_shift, int64_t N, double A, double td, double* out) {
    if (n0 < 0 || count < 0) return -1;
    int err = 0;
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < (count + 4095) / 4096; ++blk) {
        int64_t s = blk * 4096, e = s + 4096 < count ? s + 4096 : count;
        if (comb_direct(fs, fc, fo_num, fo_shift, N, A, td, n0 + s, e - s, out + s) != 0) {
            err = 1;
            continue;
        }
        for (int64_t t = s; t < e; ++t) {
            int64_t n = n0 + t;
            if (sigma != 0.0) {
                double z0, z1;
                normal_pair(seed, stream, (uint64_t)n >> 1, &z0, &z1);
                out[t] += sigma * ((n & 1) ? z1 : z0);
            }
        }
    }
    return err ? -1 : 0;
}

int synth_quantized_dy(uint64_t seed, uint32_t stream, int64_t n0, int64_t count, double sigma, int64_t fs,
                       int64_t fc, int64_t fo_num, int fo_shift, int64_t N, double A, double td, int fmt, double param,
                       void* out) {
    if (n0 < 0 || count < 0) return -1;
    if (fmt == 2 && (count % 4) != 0) return -1;
    int err = 0;
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < (count + 4095) / 4096; ++blk) {
        int64_t s = blk * 4096, e = s + 4096 < count ? s + 4096 : count;
        double x[4096];
        if (comb_direct(fs, fc, fo_num, fo_shift, N, A, td, n0 + s, e - s, x) != 0) {
            err = 1;
            continue;
        }
        uint8_t acc = 0;
        for (int64_t t = s; t < e; ++t) {
            int64_t n = n0 + t;
            double v = x[t - s];
            if (sigma != 0.0) {
                double z0, z1;
                normal_pair(seed, stream, (uint64_t)n >> 1, &z0, &z1);
                v += sigma * ((n & 1) ? z1 : z0);
            }
            if (fmt == 0) {
                ((float*)out)[t] = (float)v;
            } else if (fmt == 1) {
                ((int8_t*)out)[t] = quant8(v, param);
            } else {
                acc |= (uint8_t)(code2(v, param) << (2 * (t & 3)));
                if ((t & 3) == 3) {
                    ((uint8_t*)out)[t >> 2] = acc;
                    acc = 0;
                }
            }
        }
    }
    return err ? -1 : 0;
}
