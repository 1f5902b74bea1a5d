// Host-side plan arithmetic of libpcal: validation and the periods of the
// method (paper Sec. 2).  No CUDA call happens here, so this file is also
// what the CPU-only tests exercise through the C ABI.
#include <cmath>
#include <cstdint>

#include "pcal.h"

namespace {

int64_t gcd64(int64_t a, int64_t b) {
    while (b != 0) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a < 0 ? -a : a;
}

bool integral_hz(double v, int64_t* out) {
    if (!std::isfinite(v) || v < 0.0 || v > 9.0e15 || std::floor(v) != v) return false;
    *out = static_cast<int64_t>(v);
    return true;
}

}  // namespace

extern "C" int pcal_plan_geometry(double fs, double f_comb, double f_offset, int N, int sample_format,
                                  pcal_geometry* out) {
    int64_t ifs, ifc, ifo;
    if (!out) return PCAL_EINVAL;
    if (!integral_hz(fs, &ifs) || !integral_hz(f_comb, &ifc) || !integral_hz(f_offset, &ifo)) return PCAL_EINVAL;
    if (ifs <= 0 || ifc <= 0 || ifo >= ifc || ifs % ifc != 0) return PCAL_EINVAL;
    if (sample_format != PCAL_F32 && sample_format != PCAL_I8 && sample_format != PCAL_2BIT) return PCAL_EINVAL;
    const int64_t n_bins = ifs / ifc;  // N = fs / f_comb (text after Eq. 1)
    if (N <= 0 || static_cast<int64_t>(N) != n_bins) return PCAL_EINVAL;
    const int64_t g = gcd64(gcd64(ifs, ifc), ifo);
    const int64_t L = ifs / g;  // lcm(N_bins, N_rotator): Eq. 4 with the comb period
    if (n_bins > PCAL_MAX_N || L > PCAL_MAX_L) return PCAL_ETOOLARGE;

    pcal_geometry geo{};
    geo.fs = ifs;
    geo.f_comb = ifc;
    geo.f_offset = ifo;
    geo.N = n_bins;
    geo.N_rot = ifs / gcd64(ifs, ifo);  // Eq. 4 (gcd(fs, 0) = fs gives 1)
    geo.L = L;
    geo.step_comb = ifc / g;
    geo.step_offset = ifo / g;
    geo.format = sample_format;
    const int spw = sample_format == PCAL_F32 ? 1 : (sample_format == PCAL_I8 ? 4 : 16);
    geo.samples_per_byte_x4 = spw;
    // Bulk rows: a whole number of periods L that is also a whole number of
    // 16-byte vectors, stretched to at least 256 bytes so that every row of a
    // tile is a run of full 32-byte sectors.
    const int64_t vec = 4 * spw;  // samples per 16 bytes
    int64_t row = L / gcd64(L, vec) * vec;
    const int64_t row_bytes = row * 4 / spw;
    if (row_bytes < 256) row *= (256 + row_bytes - 1) / row_bytes;
    geo.row_samples = row;
    *out = geo;
    return PCAL_OK;
}

extern "C" const char* pcal_strerror(int code) {
    switch (code) {
        case PCAL_OK: return "success";
        case PCAL_EINVAL: return "invalid argument";
        case PCAL_ENOMEM: return "out of memory";
        case PCAL_ECUDA: return "CUDA runtime error";
        case PCAL_EBUSY: return "plan busy";
        case PCAL_ETOOLARGE: return "period L or tone count N above the library limit";
        case PCAL_ETIMEOUT: return "bounded device wait timed out";
        default: return "unknown pcal status";
    }
}
