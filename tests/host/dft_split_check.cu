// Host check of the tensor-core DFT's operand split (compiled by nvcc, run on
// the CPU; no GPU call): the words split_p_kernel's threads write form the
// same part images as splitting P element by element into the no-swizzle
// K-major layout (tile_offset), over ragged channel counts, ragged N and P at
// 8-byte (not 16-byte) alignment; the parts of every value add up to it
// within the split's precision; and the thread -> word map of each mode
// covers every word of a tile once.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dft_tc.cu"

template <int MODE>
static int check_map() {
    constexpr int kImageWords = TcCfg<MODE>::kImageWords;
    std::vector<int> seen(kImageWords, 0);
    for (int e = 0; e < kImageWords; ++e) {
        const int w = split_word_of_thread<MODE>(e);
        if (w < 0 || w >= kImageWords) return 1;
        ++seen[w];
    }
    for (int c : seen)
        if (c != 1) return 1;
    return 0;
}

// The parts of x add up to x within 2^-22 (two TF32 parts) or 2^-26 (three
// BF16 parts) of |x|, summed in double.
template <int MODE>
static int check_parts(float x) {
    uint32_t v[3];
    split_parts<MODE>(x, v);
    double s = 0;
    for (int p = 0; p < TcCfg<MODE>::kParts; ++p) s += MODE == PCAL_DFT_TC_TF32X3 ? f32_of_bits(v[p]) : f32_of_bits(v[p] << 16);
    const double tol = std::ldexp(std::fabs((double)x), MODE == PCAL_DFT_TC_TF32X3 ? -22 : -26);
    if (std::fabs(s - (double)x) > tol) {
        std::printf("mode %d: parts of %.9g add to %.17g\n", MODE, x, s);
        return 1;
    }
    return 0;
}

template <int MODE>
static int check_images(int64_t C, int N, int shift) {
    constexpr int ES = esize_of<MODE>();
    constexpr int KC = TcCfg<MODE>::kChunk / ES;
    constexpr int NP = TcCfg<MODE>::kParts;
    constexpr int kATile = TcCfg<MODE>::kATile;
    constexpr int kImageWords = TcCfg<MODE>::kImageWords;
    const int k_chunks = (2 * N + KC - 1) / KC;
    const int64_t tiles = (C + kTcM - 1) / kTcM * k_chunks;
    std::vector<float2> buf((size_t)(C * N) + 2);
    uint32_t st = 12345u + (uint32_t)(C * 131 + N);
    for (float2& v : buf) {  // values across many binades, both signs
        st = st * 1664525u + 1013904223u;
        const float a = ((int)(st >> 8) - (1 << 23)) / 8388608.0f;
        st = st * 1664525u + 1013904223u;
        v.x = a * 3.7f;
        v.y = a * ((st >> 28) + 1) * 1e-3f;
    }
    const float2* P = buf.data() + shift;
    std::vector<uint8_t> ref((size_t)tiles * NP * kATile), got((size_t)tiles * NP * kATile, 0xab);
    int bad = 0;
    for (int64_t blk = 0; blk < tiles; ++blk) {
        uint8_t* img = ref.data() + blk * NP * kATile;
        uint8_t* parts[3] = {img, img + kATile, img + 2 * kATile};
        for (int r = 0; r < kTcM; ++r)
            for (int k = 0; k < KC; ++k) {
                const int64_t c = blk / k_chunks * kTcM + r;
                const int kk = (int)(blk % k_chunks) * KC + k;
                float x = 0.f;  // [Re P | Im P], zeros past C and 2N
                if (c < C && kk < N) x = P[c * N + kk].x;
                if (c < C && kk >= N && kk < 2 * N) x = P[c * N + kk - N].y;
                const uint32_t o = tile_offset(r, k, kTcM, ES);
                split_store<MODE>(x, parts, o);
                bad += check_parts<MODE>(x);
            }
    }
    uint4* out = reinterpret_cast<uint4*>(got.data());
    for (int64_t i = 0; i < tiles * kImageWords; ++i) {  // the kernel's loop body, thread by thread
        const int64_t blk = i / kImageWords;
        const int w = split_word_of_thread<MODE>((int)(i % kImageWords));
        uint4 part[NP];
        split_word<MODE>(P, C, N, k_chunks, blk, w, part);
        for (int p = 0; p < NP; ++p) out[(blk * NP + p) * kImageWords + w] = part[p];
    }
    if (ref != got) {
        std::printf("mode %d C %lld N %d shift %d: images differ\n", MODE, (long long)C, N, shift);
        return bad + 1;
    }
    return bad;
}

int main() {
    int bad = check_map<PCAL_DFT_TC_BF16X6>() + check_map<PCAL_DFT_TC_TF32X3>();
    const int64_t Cs[] = {1, 127, 128, 300};
    const int Ns[] = {1, 3, 7, 8, 31, 64, 100, 129, 1024};
    for (int64_t C : Cs)
        for (int N : Ns)
            for (int shift = 0; shift < 2; ++shift) {
                bad += check_images<PCAL_DFT_TC_BF16X6>(C, N, shift);
                bad += check_images<PCAL_DFT_TC_TF32X3>(C, N, shift);
            }
    std::printf(bad ? "FAIL\n" : "OK\n");
    return bad ? 1 : 0;
}
