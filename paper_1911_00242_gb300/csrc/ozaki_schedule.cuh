// Schedule of the Ozaki GEMM's work within one output tile: the exact TMEM windows
// and the split of a tile's (chunk, diagonal) units over CTAs.  Host-callable as well,
// so that the CPU tests check this code itself.
#pragma once
#include <cuda_runtime.h>

namespace ccsdk {

// stages (64 K each) per exact TMEM window of diagonal d
__host__ __device__ constexpr int oz_win(int d) { return d == 0 ? 16 : 32; }

// Work of one tile, in units u = c * s + d (chunk c, diagonal d = p + q of the slice
// pairs), each (d + 1) * kstages stages.  With nsplit > 1, CTA `split` takes the units
// whose first stage lies in its share [split, split + 1) * total / nsplit of the stages.
__host__ __device__ __forceinline__ void oz_unit_range(int nch, int S, int kstages, int nsplit, int split, int& u0, int& u1) {
    const int nunits = nch * S;
    if (nsplit <= 1) { u0 = 0; u1 = nunits; return; }
    const long long per_chunk = (long long)(S * (S + 1) / 2) * kstages;
    const long long total = per_chunk * nch;
    const long long lo = total * split / nsplit, hi = total * (split + 1) / nsplit;
    u0 = nunits; u1 = nunits;
    for (int u = 0; u < nunits; ++u) {
        const int c = u / S, d = u - (u / S) * S;
        const long long start = c * per_chunk + (long long)(d * (d + 1) / 2) * kstages;
        if (start >= lo && u0 == nunits) u0 = u;
        if (start >= hi) { u1 = u; break; }
    }
    if (u1 < u0) u1 = u0;
}

}  // namespace ccsdk
