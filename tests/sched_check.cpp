// Property checks of the persistent launch's host scheduling rules (tail split,
// download bands); compiled and run by test_schedule_host.py on the CPU.
#include <stdio.h>

#include <vector>

#include "../paper_2512_18010_b300/csrc/tc_schedule.h"

using namespace scff::sched;

#define CHECK(c, ...)                                      \
    do {                                                   \
        if (!(c)) {                                        \
            printf("FAIL line %d: ", __LINE__);            \
            printf(__VA_ARGS__);                           \
            printf("\n");                                  \
            return 1;                                      \
        }                                                  \
    } while (0)

static double tail_len(int r, int c, int P) { return (double)((r * c + P - 1) / P) / c; }

static bool allowed(int r, int c, int nkc, int P) {
    return r > 0 && nkc < 32768 && c >= 2 && c <= 16 && c <= nkc / 8 && (long long)r * c <= 2LL * P;
}

int main() {
    const int P = 148;
    // ---- tail split: the chosen s is allowed, shortens the tail below one tile
    // time, and no allowed part count gives a shorter tail (brute force)
    const int nkcs[] = {1, 8, 15, 16, 40, 100, 1025, 40000};
    for (int items = 1; items <= 3000; ++items)
        for (int nkc : nkcs) {
            int R = -1, s = -1;
            tail_split(items, nkc, P, &R, &s);
            const int r = items % P;
            double best = 1.0;
            for (int c = 2; c <= 16; ++c)
                if (allowed(r, c, nkc, P) && tail_len(r, c, P) < best) best = tail_len(r, c, P);
            if (s == 0) {
                CHECK(R == 0, "items %d nkc %d: unsplit tail reports R = %d", items, nkc, R);
                CHECK(best >= 1.0 - 1e-12, "items %d nkc %d: a split would shorten the tail", items, nkc);
            } else {
                CHECK(R == r, "items %d: R %d", items, R);
                CHECK(allowed(r, s, nkc, P), "items %d nkc %d: s %d not allowed", items, nkc, s);
                CHECK(tail_len(r, s, P) < 1.0, "items %d: tail %g", items, tail_len(r, s, P));
                CHECK(tail_len(r, s, P) <= best + 1e-12, "items %d: s %d not optimal", items, s);
            }
        }
    // ---- bands: every column tile in exactly one band, mirrored pairs together,
    // boundaries increasing; automatic bands end at wave ends
    const int reqs[] = {0, 1, 2, 3, 5, 8};
    for (int n_mt = 1; n_mt <= 7; ++n_mt)
        for (int n_nt = 1; n_nt <= 160; ++n_nt)
            for (int mirror = 0; mirror < 2; ++mirror)
                for (int req : reqs) {
                    const long long tiles = (long long)n_mt * n_nt;
                    int R = 0, s = 0;
                    tail_split((int)tiles, 200, P, &R, &s);
                    const long long first_split = s ? tiles - R : tiles;
                    const long long n_items = first_split + (tiles - first_split) * (s ? s : 1);
                    const int grid = (int)(n_items < P ? n_items : P);
                    int b[9];
                    const int G = band_bounds(n_mt, n_nt, mirror != 0, (long long)n_nt * 128, 128, req, grid,
                                              first_split, s, 8, b);
                    const int D = mirror ? (n_nt + 1) / 2 : n_nt;
                    if (req == 1) CHECK(G == 1, "banding not off");
                    if (G == 1) continue;
                    CHECK(G >= 2 && G <= 8, "G %d", G);
                    CHECK(b[0] == 0 && b[G] == D, "ends %d %d (D %d)", b[0], b[G], D);
                    std::vector<int> owner(n_nt, -1);
                    for (int g = 0; g < G; ++g) {
                        CHECK(b[g + 1] > b[g], "bounds not increasing");
                        int runs[2][2];
                        const int nr = band_runs(n_nt, mirror != 0, b[g], b[g + 1], runs);
                        for (int q = 0; q < nr; ++q)
                            for (int nt = runs[q][0]; nt < runs[q][1]; ++nt) {
                                CHECK(nt >= 0 && nt < n_nt, "tile %d out of range", nt);
                                CHECK(owner[nt] < 0, "tile %d in two bands", nt);
                                owner[nt] = g;
                            }
                    }
                    for (int nt = 0; nt < n_nt; ++nt) {
                        CHECK(owner[nt] >= 0, "n_mt %d n_nt %d mirror %d req %d: tile %d in no band", n_mt, n_nt,
                              mirror, req, nt);
                        if (mirror) CHECK(owner[nt] == owner[n_nt - 1 - nt], "mirror pair split");
                    }
                    if (req == 0) {
                        auto item_end = [&](int e) {
                            const long long t = n_mt * band_cols(n_nt, mirror != 0, e);
                            return t <= first_split ? t : first_split + (t - first_split) * s;
                        };
                        for (int g = 1; g < G; ++g) {
                            // b[g] is the last d boundary at or below some wave end k * grid
                            const long long k = (item_end(b[g]) + grid - 1) / grid;
                            bool ok = false;
                            for (long long kk = k; kk <= k + 1 && !ok; ++kk)
                                ok = item_end(b[g]) <= kk * grid && item_end(b[g] + 1) > kk * grid;
                            CHECK(ok, "n_mt %d n_nt %d: band end %d not at a wave end", n_mt, n_nt, b[g]);
                        }
                    }
                }
    // mirrored columns that straddle tiles: no banding
    {
        int b[9];
        CHECK(band_bounds(6, 128, true, 128LL * 128 - 5, 128, 0, P, 740, 5, 8, b) == 1, "ragged mirror banded");
    }
    printf("ok\n");
    return 0;
}
