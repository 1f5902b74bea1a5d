// Host check of the bit-sliced counting used by the 2-bit bulk kernel:
// Harley-Seal accumulation + ripple + (h AND l) packing + 16x16x2 transpose
// against plain per-bit counting, on random words and on all-ones words.
#include <cstdio>
#include <cstdint>
#include <random>

#include "bitplane.cuh"

static uint32_t d3_unused() { return 0; }

template <int U>
int run(uint64_t seed, int blocks, bool all_ones) {
    std::mt19937_64 rng(seed);
    uint32_t w1 = 0, w2 = 0, w4 = 0, w8 = 0, w16 = 0, wu[U] = {0};
    uint32_t d1 = 0, d2 = 0, d4 = 0, d8 = 0, du[U] = {0};
    uint64_t ref_l[16] = {0}, ref_h[16] = {0}, ref_hl[16] = {0};
    for (int b = 0; b < blocks; ++b) {
        uint32_t x[32];
        for (int i = 0; i < 32; ++i) {
            x[i] = all_ones ? 0xFFFFFFFFu : (uint32_t)rng();
            for (int j = 0; j < 16; ++j) {
                uint32_t c = (x[i] >> (2 * j)) & 3u;
                ref_l[j] += c & 1u;
                ref_h[j] += c >> 1;
                ref_hl[j] += (c == 3u);
            }
        }
        pcal_bits::add32<U>(x, w1, w2, w4, w8, w16, wu, d1, d2, d4, d8, du);
    }
    uint32_t W[16] = {w1, w2, w4, w8, w16}, D[16] = {d1, d2, d3_unused(), d8};
    D[2] = d4;
    for (int u = 0; u < U; ++u) {
        if (5 + u < 16) W[5 + u] = wu[u];
        if (4 + u < 16) D[4 + u] = du[u];
    }
    for (int i = 5 + U; i < 16; ++i) W[i] = 0;
    for (int i = 4 + U; i < 16; ++i) D[i] = 0;
    pcal_bits::transpose16x2(W);
    pcal_bits::transpose16x2(D);
    auto lane = [](const uint32_t* A, int p) { return (A[p & 15] >> (16 * (p >> 4))) & 0xFFFFu; };
    int bad = 0;
    for (int j = 0; j < 16; ++j) {
        uint64_t l = lane(W, 2 * j), h = lane(W, 2 * j + 1), hl = lane(D, 2 * j) + lane(D, 2 * j + 1);
        if (l != ref_l[j] || h != ref_h[j] || hl != ref_hl[j]) {
            if (bad < 5)
                std::printf("U=%d blocks=%d j=%d: l %llu/%llu h %llu/%llu hl %llu/%llu\n", U, blocks, j,
                            (unsigned long long)l, (unsigned long long)ref_l[j], (unsigned long long)h,
                            (unsigned long long)ref_h[j], (unsigned long long)hl, (unsigned long long)ref_hl[j]);
            ++bad;
        }
    }
    return bad;
}

int main() {
    int bad = 0;
    for (int s = 0; s < 20; ++s) {
        bad += run<3>(s, 3, false);
        bad += run<5>(100 + s, 31, false);
        bad += run<7>(200 + s, 127, false);
        bad += run<9>(300 + s, 300, false);
        bad += run<11>(400 + s, 700, false);
    }
    // largest counts each template supports: every bit set in every word
    bad += run<3>(1, 7, true);
    bad += run<5>(1, 31, true);
    bad += run<11>(1, 2047, true);
    std::printf(bad ? "FAIL %d\n" : "OK\n", bad);
    return bad != 0;
}
