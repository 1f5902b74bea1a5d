// Host check of the server's HBM arena against a brute-force model (one flag
// per 256-byte unit): over random alloc / release sequences, alloc returns
// the lowest-offset free run that fits (first fit), fails exactly when no run
// fits, never overlaps a live block; used() counts the live units; free blocks
// stay coalesced (one per maximal free run); releasing everything leaves one
// free block of the full size.
#include <cstdio>
#include <random>
#include <vector>

#include "arena.h"

using pcal_arena::Arena;
using pcal_arena::kGrain;

struct Live {
    size_t off, bytes;
};

static int fail(const char* what, int step) {
    std::printf("step %d: %s\n", step, what);
    return 1;
}

static int run(uint64_t seed, size_t units, int steps) {
    std::mt19937_64 rng(seed);
    Arena a;
    a.reset(units * kGrain);
    std::vector<char> busy(units, 0);
    std::vector<Live> live;
    for (int s = 0; s < steps; ++s) {
        if (live.empty() || rng() % 100 < 55) {
            const size_t bytes = 1 + rng() % (units * kGrain / 6);  // not a multiple of the grain
            const size_t need = (bytes + kGrain - 1) / kGrain;
            size_t expect = units, run_len = 0;  // first free run of >= need units
            for (size_t u = 0; u < units && expect == units; ++u) {
                run_len = busy[u] ? 0 : run_len + 1;
                if (run_len == need) expect = u + 1 - need;
            }
            size_t off = ~(size_t)0;
            const bool ok = a.alloc(bytes, &off);
            if (ok != (expect != units)) return fail("alloc success differs from the model", s);
            if (!ok) continue;
            if (off != expect * kGrain) return fail("not the first fit", s);
            for (size_t u = expect; u < expect + need; ++u) {
                if (busy[u]) return fail("overlaps a live block", s);
                busy[u] = 1;
            }
            live.push_back({off, bytes});
        } else {
            const size_t i = rng() % live.size();
            a.release(live[i].off, live[i].bytes);
            const size_t u0 = live[i].off / kGrain, n = (live[i].bytes + kGrain - 1) / kGrain;
            for (size_t u = u0; u < u0 + n; ++u) busy[u] = 0;
            live[i] = live.back();
            live.pop_back();
        }
        size_t used = 0, runs = 0;
        for (size_t u = 0; u < units; ++u) {
            used += busy[u];
            runs += !busy[u] && (u == 0 || busy[u - 1]);
        }
        if (a.used() != used * kGrain) return fail("used() differs", s);
        if (a.free_blocks() != runs) return fail("free blocks not coalesced", s);
    }
    for (const Live& l : live) a.release(l.off, l.bytes);
    if (a.used() != 0 || a.free_blocks() != 1) return fail("not whole after releasing everything", steps);
    size_t off = 1;
    if (!a.alloc(units * kGrain, &off) || off != 0) return fail("full-size block not available", steps);
    return 0;
}

int main() {
    int bad = 0;
    for (uint64_t seed = 1; seed <= 20; ++seed) bad += run(seed, 64 + seed * 37, 3000);
    Arena e;
    e.reset(0);
    size_t off = 0;
    bad += e.alloc(1, &off) ? fail("empty arena gave a block", 0) : 0;
    std::printf(bad ? "FAIL\n" : "OK\n");
    return bad ? 1 : 0;
}
