// Randomised check of the device-pool arena (host code only): every range it
// hands out is aligned, inside the pool and disjoint from the others; it is
// the lowest-addressed free gap that fits (first fit, computed here by brute
// force from the live ranges); after everything is freed the pool is one
// range again. Prints "OK <operations>" or the first violation.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>

#include "../../paper_1204_6734_gb300/csrc/flb_arena.h"

int main(int argc, char** argv) {
    const unsigned seed = argc > 1 ? (unsigned)atoi(argv[1]) : 1u;
    std::mt19937_64 rng(seed);
    const size_t pool = (size_t)1 << 30;
    flb::Arena a(pool);
    std::map<size_t, size_t> live;   // offset -> rounded size
    long ops = 0;
    for (int it = 0; it < 200000; ++it) {
        const bool do_alloc = live.empty() || (rng() % 100) < 55;
        if (do_alloc) {
            const size_t bytes = 1 + rng() % (size_t)(8u << 20);
            const size_t need = flb::Arena::round_up(bytes);
            // brute-force first fit over the gaps between live ranges
            size_t expect = (size_t)-1, cur = 0;
            for (auto& kv : live) {
                if (kv.first - cur >= need) { expect = cur; break; }
                cur = kv.first + kv.second;
            }
            if (expect == (size_t)-1 && pool - cur >= need) expect = cur;
            size_t off = 0;
            const bool ok = a.alloc(bytes, &off);
            if (ok != (expect != (size_t)-1) || (ok && off != expect)) {
                printf("FAIL first fit at op %ld: got %d %zu expected %zu\n", ops, ok, off, expect);
                return 1;
            }
            if (ok) {
                if (off % flb::Arena::kAlign || off + need > pool) {
                    printf("FAIL bounds/alignment at op %ld\n", ops);
                    return 1;
                }
                live[off] = need;
            }
        } else {
            auto it2 = live.begin();
            std::advance(it2, rng() % live.size());
            if (!a.release(it2->first)) {
                printf("FAIL release at op %ld\n", ops);
                return 1;
            }
            live.erase(it2);
            if (a.release((size_t)3 + (rng() % 1000) * flb::Arena::kAlign)) {   // never a range start
                printf("FAIL released a non-range at op %ld\n", ops);
                return 1;
            }
        }
        size_t used = 0;
        for (auto& kv : live) used += kv.second;
        if (used != a.used() || a.live_ranges() != live.size()) {
            printf("FAIL accounting at op %ld\n", ops);
            return 1;
        }
        ++ops;
    }
    for (auto& kv : live) a.release(kv.first);
    if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != pool) {
        printf("FAIL not coalesced: %zu ranges\n", a.free_ranges());
        return 1;
    }
    printf("OK %ld\n", ops);
    return 0;
}
