// Host-side scheduling rules of the persistent tensor-core launch: the tail
// split of a job's last partial wave and the output-column bands of the
// overlapped download.  Plain C++ (no CUDA types), so the rules are also
// compiled and checked on a machine without a GPU.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace scff {
namespace sched {

// Tail split of a job with `items` equal tiles of nkc chunks on P SMs: the
// last R = items mod P tiles run as s parts (k split evenly), so that the
// final wave keeps the SMs busy.  s (2..16, parts of at least 8 chunks, at
// most 2P parts in all) minimises the tail's length ceil(R s / P) / s in tile
// times; when no s gets it below one tile time the tail is not split
// (R = s = 0).
inline void tail_split(int items, int nkc, int P, int *R, int *s) {
    *R = items % P;
    *s = 0;
    if (nkc >= 32768) *R = 0;  // the k0 field of a work item holds 15 bits
    if (*R == 0) return;
    double best = 1.0;
    for (int c = 2; c <= 16 && c <= nkc / 8 && (int64_t)*R * c <= 2 * (int64_t)P; ++c) {
        const double t = (double)((*R * c + P - 1) / P) / c;
        if (t < best - 1e-9) {
            best = t;
            *s = c;
        }
    }
    if (!*s) *R = 0;
}

// Runs of n-tiles [runs[i][0], runs[i][1]) of the band [d0, d1).  With the
// mirror, tile nt and its mirror n_nt-1-nt (which receives nt's mirrored
// columns when N is a multiple of the tile width) belong to the same band:
// bands are ranges of d = min(nt, n_nt-1-nt).  Without it d = nt.  Returns
// the number of runs (0..2).
inline int band_runs(int n_nt, bool mirror, int d0, int d1, int runs[2][2]) {
    if (!mirror) {
        runs[0][0] = d0;
        runs[0][1] = d1;
        return d1 > d0 ? 1 : 0;
    }
    int n = 0;
    if (d1 > d0) {
        runs[n][0] = d0;
        runs[n][1] = d1;
        ++n;
    }
    const int lo = std::max(n_nt - d1, d1), hi = n_nt - d0;
    if (hi > lo) {
        runs[n][0] = lo;
        runs[n][1] = hi;
        ++n;
    }
    return n;
}

// Column tiles of the d values below e: 2e with the mirror (one for the
// middle tile of an odd n_nt), else e.
inline int64_t band_cols(int n_nt, bool mirror, int e) {
    return mirror ? std::min(2 * (int64_t)e, (int64_t)n_nt) : e;
}

// Band boundaries 0 = b[0] < ... < b[G] = D in d units (D = ceil(n_nt / 2)
// with the mirror, else n_nt) for the band-major tile order of one launch on
// `grid` CTAs; returns G (1: no banding).  b must hold max_bands + 1 entries.
// A requested count (2..max_bands) gives equal bands; 1 turns banding off.
// Automatic (requested = 0; jobs of at least 1.25 waves): CTA c runs items
// c, c + grid, ..., so the items below k * grid are all written when wave k
// ends; the bands end at the last d boundary below each wave end (the last
// max_bands - 1 of them), so each band's copy starts one wave after its first
// tiles and only the last wave's columns (less the tail split's time) wait
// for the launch to end.  first_split, nsplit: the tail split of the job's
// tile count (the items of tile t >= first_split are its nsplit parts).
// With the mirror, N (columns) must be a multiple of the tile width bn, else
// mirrored columns would straddle tiles and banding is off.
inline int band_bounds(int n_mt, int n_nt, bool mirror, int64_t N, int bn, int requested, int grid,
                       int64_t first_split, int nsplit, int max_bands, int *b) {
    if (requested == 1 || n_mt <= 0 || n_nt <= 0) return 1;
    if (mirror && N % bn) return 1;
    const int D = mirror ? (n_nt + 1) / 2 : n_nt;
    int G = 0;
    b[0] = 0;
    if (requested > 0) {
        G = std::min(std::min(requested, max_bands), D);
        for (int g = 1; g <= G; ++g) b[g] = (int)((int64_t)g * D / G);
        return G >= 2 ? G : 1;
    }
    const int64_t tiles = (int64_t)n_mt * n_nt;
    if (tiles * 4 < 5 * (int64_t)grid) return 1;
    auto item_end = [&](int e) {
        const int64_t t = n_mt * band_cols(n_nt, mirror, e);
        return t <= first_split ? t : first_split + (t - first_split) * nsplit;
    };
    std::vector<int> ends;  // d boundaries at wave ends, increasing
    for (int64_t k = 1; item_end(D) > k * grid; ++k) {
        int e = ends.empty() ? 0 : ends.back();
        while (e < D && item_end(e + 1) <= k * grid) ++e;
        if (e > (ends.empty() ? 0 : ends.back())) ends.push_back(e);
    }
    const int keep = std::min((int)ends.size(), max_bands - 1);
    for (int i = (int)ends.size() - keep; i < (int)ends.size(); ++i) b[++G] = ends[i];
    b[++G] = D;
    return G >= 2 ? G : 1;
}

}  // namespace sched
}  // namespace scff
