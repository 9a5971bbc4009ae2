// Schedule of the Ozaki GEMM's work within one output tile: the exact TMEM windows
// and the split of a tile's (chunk, window) units over CTAs.  Host-callable as well,
// so that the CPU tests check this code itself.
#pragma once
#include <cuda_runtime.h>

namespace ccsdk {

// K slices (64 K each) per exact TMEM window with s slices.  One window sums, for every
// diagonal d = p + q at once, the products of all its pairs over the window's K.  The
// digits obey |v_0| <= 128 and |v_p| <= 64 (p >= 1), so per K element diagonal 0 adds
// at most 2^14 and diagonal d >= 1 at most 2 * 2^13 (pairs (0, d), (d, 0)) plus
// (d - 1) * 2^12 (the others) = 2^12 (d + 3), largest at d = s - 1.  Keeping every
// partial sum within 2^24 (exact in FP32) allows 64 / (s + 2) slices of 64 K for the
// diagonals d >= 1 and 16 for diagonal 0.
__host__ __device__ constexpr int oz_kwin(int s) { return s <= 1 ? 16 : (64 / (s + 2) < 16 ? 64 / (s + 2) : 16); }

// Windows of one chunk of kstages K slices.
__host__ __device__ constexpr int oz_nwin(int kstages, int s) { return (kstages + oz_kwin(s) - 1) / oz_kwin(s); }

// Work of one tile, in units u = c * nw + wi (chunk c, window wi of nw = oz_nwin per
// chunk), window wi covering K slices [wi W, min((wi + 1) W, kstages)).  With nsplit > 1,
// CTA `split` takes the units whose first K slice lies in its share
// [split, split + 1) * total / nsplit of the tile's K slices.
__host__ __device__ __forceinline__ void oz_unit_range(int nch, int S, int kstages, int nsplit, int split, int& u0, int& u1) {
    const int W = oz_kwin(S), nw = oz_nwin(kstages, S);
    const int nunits = nch * nw;
    if (nsplit <= 1) { u0 = 0; u1 = nunits; return; }
    const long long total = (long long)nch * kstages;
    const long long lo = total * split / nsplit, hi = total * (split + 1) / nsplit;
    u0 = nunits; u1 = nunits;
    for (int u = 0; u < nunits; ++u) {
        const int c = u / nw, wi = u - (u / nw) * nw;
        const long long start = (long long)c * kstages + (long long)wi * W;
        if (start >= lo && u0 == nunits) u0 = u;
        if (start >= hi) { u1 = u; break; }
    }
    if (u1 < u0) u1 = u0;
}

}  // namespace ccsdk
