// Host check of the double-float arithmetic used by the finalize kernels:
// add, multiply, divide, square root and accumulation against FP64, on
// random operands spanning many magnitudes.
#include <cmath>
#include <cstdio>
#include <random>

#include "df64.cuh"

using pcal_df::df;

static df split(double x) {
    float hi = (float)x;
    return df{hi, (float)(x - (double)hi)};
}
static double val(df x) { return (double)x.hi + (double)x.lo; }

int main() {
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    std::uniform_int_distribution<int> e(-20, 20);
    int bad = 0;
    double worst[5] = {0, 0, 0, 0, 0};
    for (int it = 0; it < 200000; ++it) {
        double a = std::ldexp(u(rng), e(rng)), b = std::ldexp(u(rng), e(rng));
        df A = split(a), B = split(b);
        // reference on the exact df inputs
        double ra = val(A), rb = val(B);
        double r[5] = {ra + rb, ra * rb, rb != 0 ? ra / rb : 0.0, std::sqrt(std::fabs(ra)), 0.0};
        df got[5] = {pcal_df::add(A, B), pcal_df::mul(A, B), rb != 0 ? pcal_df::div(A, B) : df{0, 0},
                     pcal_df::sqrt_df(df{std::fabs(A.hi), A.hi < 0 ? -A.lo : A.lo}), df{0, 0}};
        for (int k = 0; k < 4; ++k) {
            double scale = k == 0 ? std::fmax(std::fabs(ra), std::fabs(rb)) : std::fabs(r[k]);
            if (scale == 0) continue;
            double err = std::fabs(val(got[k]) - r[k]) / scale;
            if (err > worst[k]) worst[k] = err;
        }
    }
    // long accumulation: 1e6 terms of mixed sign
    df acc{0, 0};
    long double ref = 0;
    for (int i = 0; i < 1000000; ++i) {
        float x = (float)std::ldexp(u(rng), e(rng) / 4);
        acc = pcal_df::add_f(acc, x);
        ref += x;
    }
    worst[4] = std::fabs(val(acc) - (double)ref) / 1000000.0;
    const double lim[5] = {1e-13, 1e-13, 1e-13, 1e-13, 1e-12};
    const char* names[5] = {"add", "mul", "div", "sqrt", "accumulate"};
    for (int k = 0; k < 5; ++k) {
        std::printf("%-10s worst rel err %.3g\n", names[k], worst[k]);
        if (!(worst[k] < lim[k])) ++bad;
    }
    std::printf(bad ? "FAIL\n" : "OK\n");
    return bad != 0;
}
