// Bit-sliced counters for the 2-bit fold.
//
// A 32-bit word of 2-bit samples holds 16 samples; bit 2j is the l bit and
// bit 2j+1 the h bit of sample j (code = (h<<1)|l).  A thread that always
// reads the SAME word position of every row sees the same 16 bins in every
// word, so it can count, for each of the 32 bit positions, how many of its
// words have that bit set -- a "positional popcount".  It keeps the counts
// bit-sliced: plane i holds bit i of all 32 counters, and adding a word is a
// carry-save (full-adder) operation on whole planes, two 3-input logic ops
// per full adder for all 32 counters at once.  Words are added 16 at a time
// through a Harley-Seal tree (15 full adders), whose weight-16 output ripples
// into the upper planes.
//
// The h AND l count of each sample comes from a second stream: for a pair of
// words (a, b), d = (a & (a>>1) & 0x5555...) | (b & (b<<1) & 0xAAAA...) puts
// the (h AND l) bit of sample j of word a at bit 2j and that of word b at bit
// 2j+1, so one word of the second stream counts two input words.
//
// At the end the planes are turned into integers by a bit-matrix transpose
// of 16 planes x 32 positions done as two independent 16x16 transposes (low
// and high half of each word): afterwards word i holds the count of position
// i in its low 16 bits and of position i+16 in its high 16 bits.
#pragma once

#include <stdint.h>

#ifndef PCAL_HD
#if defined(__CUDACC__)
#define PCAL_HD __host__ __device__ __forceinline__
#else
#define PCAL_HD inline
#endif
#endif

namespace pcal_bits {

// Three-input logic op: one LOP3 on the device (lut over a=0xF0, b=0xCC,
// c=0xAA), the plain expression on the host.
template <int LUT>
PCAL_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
#else
    uint32_t d = 0;
    for (int bit = 0; bit < 32; ++bit) {
        const int idx = (((a >> bit) & 1) << 2) | (((b >> bit) & 1) << 1) | ((c >> bit) & 1);
        d |= (uint32_t)((LUT >> idx) & 1) << bit;
    }
    return d;
#endif
}
constexpr int kXor3 = 0x96;  // a ^ b ^ c
constexpr int kMaj3 = 0xE8;  // majority(a, b, c)

// Full adder on bit planes: l = a ^ b ^ c, h = majority(a, b, c).
PCAL_HD void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t hh = lop3<kMaj3>(a, b, c);
    l = lop3<kXor3>(a, b, c);
    h = hh;
}

// Adds 16 words into (ones, twos, fours, eights); returns the weight-16 carry.
PCAL_HD uint32_t harley_seal16(const uint32_t* x, uint32_t& ones, uint32_t& twos, uint32_t& fours, uint32_t& eights) {
    uint32_t tA, tB, fA, fB, eA, eB, s16;
    csa(tA, ones, ones, x[0], x[1]);
    csa(tB, ones, ones, x[2], x[3]);
    csa(fA, twos, twos, tA, tB);
    csa(tA, ones, ones, x[4], x[5]);
    csa(tB, ones, ones, x[6], x[7]);
    csa(fB, twos, twos, tA, tB);
    csa(eA, fours, fours, fA, fB);
    csa(tA, ones, ones, x[8], x[9]);
    csa(tB, ones, ones, x[10], x[11]);
    csa(fA, twos, twos, tA, tB);
    csa(tA, ones, ones, x[12], x[13]);
    csa(tB, ones, ones, x[14], x[15]);
    csa(fB, twos, twos, tA, tB);
    csa(eB, fours, fours, fA, fB);
    csa(s16, eights, eights, eA, eB);
    return s16;
}

// Adds 8 words into (ones, twos, fours); returns the weight-8 carry.
PCAL_HD uint32_t harley_seal8(const uint32_t* x, uint32_t& ones, uint32_t& twos, uint32_t& fours) {
    uint32_t tA, tB, fA, fB, e8;
    csa(tA, ones, ones, x[0], x[1]);
    csa(tB, ones, ones, x[2], x[3]);
    csa(fA, twos, twos, tA, tB);
    csa(tA, ones, ones, x[4], x[5]);
    csa(tB, ones, ones, x[6], x[7]);
    csa(fB, twos, twos, tA, tB);
    csa(e8, fours, fours, fA, fB);
    return e8;
}

// Ripple-carry increment of a U-plane counter by the 1-bit word x.
template <int U>
PCAL_HD void ripple(uint32_t (&up)[U], uint32_t x) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t c = up[u] & x;
        up[u] ^= x;
        x = c;
    }
}

// (h AND l) bits of two words packed into one (see the header comment).
PCAL_HD uint32_t hl_pair(uint32_t a, uint32_t b) {
    const uint32_t x = lop3<0x80>(a, a >> 1, 0x55555555u);  // a & (a>>1) & mask
    const uint32_t y = b & (b + b);                          // hl of b at odd bits
    return lop3<0xF8>(x, y, 0xAAAAAAAAu);                   // x | (y & mask)
}

// Thirty-two words of one column: the w stream (l and h bits) through two
// Harley-Seal trees and one full adder at weight 16, the (h AND l) stream
// through one tree on the 16 packed words.  Returns nothing; the carries of
// weight 32 (w) and 16 (d) ripple into the upper planes.
template <int U>
PCAL_HD void add32(const uint32_t* x, uint32_t& w1, uint32_t& w2, uint32_t& w4, uint32_t& w8, uint32_t& w16,
                   uint32_t (&wu)[U], uint32_t& d1, uint32_t& d2, uint32_t& d4, uint32_t& d8, uint32_t (&du)[U]) {
    uint32_t d[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) d[m] = hl_pair(x[2 * m], x[2 * m + 1]);
    const uint32_t a = harley_seal16(x, w1, w2, w4, w8);
    const uint32_t b = harley_seal16(x + 16, w1, w2, w4, w8);
    uint32_t c32;
    csa(c32, w16, w16, a, b);
    ripple<U>(wu, c32);
    ripple<U>(du, harley_seal16(d, d1, d2, d4, d8));
}

// In-place transpose of two 16x16 bit matrices held in the low and high
// halves of A[0..15]: afterwards bit b of A[i] (low half) is the former bit
// i of A[b], and likewise for the high half with i+16.
PCAL_HD void transpose16x2(uint32_t (&A)[16]) {
#pragma unroll
    for (int j = 8, s = 0; j > 0; j >>= 1, ++s) {
        const uint32_t m = s == 0 ? 0x00FF00FFu : (s == 1 ? 0x0F0F0F0Fu : (s == 2 ? 0x33333333u : 0x55555555u));
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (r & j) continue;
            const uint32_t t = ((A[r] >> j) ^ A[r + j]) & m;
            A[r] ^= t << j;
            A[r + j] ^= t;
        }
    }
}

}  // namespace pcal_bits
