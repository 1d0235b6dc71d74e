// Host-side check of the balanced work partition shared by the mixing, FFT and moving-source
// kernels and the reduction (struct Partition): it compiles the library's own header and
// replays, on the CPU, the order in which a CTA walks its units and flushes its runs.
// Prints "ok" or the first violated property; no GPU is used.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "common.cuh"

using hrir::Partition;

static int fail(const char *what, long long a, long long b, long long c, long long d)
{
    std::printf("FAIL %s (%lld %lld %lld %lld)\n", what, a, b, c, d);
    return 1;
}

// One case: n_tiles tiles x n_src sources over P CTAs, runs of at most gs sources.
static int check(int n_tiles, int n_src, long long P_req, int gs)
{
    Partition p;
    p.U = (int64_t)n_tiles * n_src;
    p.P = P_req < p.U ? P_req : p.U;
    p.n_src = n_src;
    p.gs = gs;
    if (p.first(0) != 0 || p.first(p.P) != p.U) return fail("range ends", n_tiles, n_src, p.P, gs);
    const int64_t q = p.U / p.P;
    for (int64_t b = 0; b < p.P; ++b) {
        const int64_t n = p.first(b + 1) - p.first(b);
        if (n != q && n != q + 1) return fail("balance", n_tiles, n_src, p.P, b);
    }
    for (int64_t u = 0; u < p.U; ++u) {
        const int64_t o = p.owner(u);
        if (o < 0 || o >= p.P || p.first(o) > u || u >= p.first(o + 1))
            return fail("owner", n_tiles, n_src, p.P, u);
    }
    // replay the kernels' walk: CTA b accumulates its units in order; a run is written out
    // (flushed) after gs units or at the end of the CTA's units in a tile, into the next slot
    // from slot_base(b, tile).  A unit belongs to the slot its run is flushed into.
    std::vector<std::vector<int>> slot_of(n_tiles, std::vector<int>(n_src, -1));
    for (int64_t b = 0; b < p.P; ++b) {
        const int64_t u0 = p.first(b), u1 = p.first(b + 1);
        int t = (int)(u0 / n_src), s = (int)(u0 % n_src);
        int slot = p.slot_base(b, t), run_n = 0;
        std::vector<int> pending;                 // sources of the run being accumulated
        for (int64_t u = u0; u < u1; ++u) {
            pending.push_back(s);
            ++run_n;
            const bool tile_end = (u + 1 == u1) || (s + 1 == n_src);
            if (run_n == gs || tile_end) {
                for (int ps : pending) slot_of[t][ps] = slot;
                pending.clear();
                ++slot;
                run_n = 0;
            }
            if (++s == n_src) {
                s = 0;
                ++t;
                if (u + 1 < u1) slot = p.slot_base(b, t);
            }
        }
    }
    for (int t = 0; t < n_tiles; ++t) {
        const int ns = p.slots(t);
        std::vector<int> count(ns > 0 ? ns : 1, 0);
        int prev = -1;
        for (int s = 0; s < n_src; ++s) {
            const int sl = slot_of[t][s];
            if (sl < 0 || sl >= ns) return fail("slot range", t, s, sl, ns);
            if (sl < prev) return fail("slot order", t, s, sl, prev);   // slots follow source order
            prev = sl;
            ++count[sl];
        }
        for (int k = 0; k < ns; ++k)
            if (count[k] < 1 || count[k] > gs) return fail("run size", t, k, count[k], gs);
    }
    return 0;
}

int main()
{
    const int tiles[] = {1, 2, 3, 7, 73};
    const int srcs[] = {1, 2, 5, 31, 64, 65, 300, 1024};
    const long long ctas[] = {1, 2, 7, 152, 304, 100000};
    const int runs[] = {1, 4, 32, 64};
    int n = 0;
    for (int t : tiles)
        for (int s : srcs)
            for (long long c : ctas)
                for (int g : runs) {
                    if (check(t, s, c, g)) return 1;
                    ++n;
                }
    std::printf("ok %d cases\n", n);
    return 0;
}
