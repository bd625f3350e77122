// Host-side split of a galaxy catalogue over processes, one per GPU.  Galaxies
// are independent units of the method (Sec. 4 fits them in parallel with no
// exchange), so a catalogue splits into contiguous blocks.  The cost of a
// gradient evaluation is a fixed part (SFH quadrature, burst, MDF) plus a part
// that grows with the galaxy's observed bands (one c_SSP row each), so a galaxy
// weighs base + popcount(mask).  The split minimises the heaviest block: binary
// search on the bound T with a greedy feasibility scan, exact for integer
// weights.  A block is also cut once the galaxies left are no more than the
// blocks left, so every block holds a galaxy while there are enough of them
// (and each galaxy its own block when there are fewer); a single galaxy never
// exceeds T, so these cuts keep the bound.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/sps.h"

namespace sps {
void set_last_error(const char* msg);
}

namespace {

int popcount32(uint32_t v) {
    int c = 0;
    for (; v; v &= v - 1) ++c;
    return c;
}

// Number of blocks the greedy scan needs under bound T (every w <= T).
int64_t blocks_needed(const std::vector<int64_t>& w, int64_t T) {
    int64_t blocks = 1, cur = 0;
    for (int64_t x : w) {
        if (cur + x > T) {
            ++blocks;
            cur = x;
        } else {
            cur += x;
        }
    }
    return blocks;
}

}  // namespace

extern "C" sps_status sps_partition_galaxies(const uint32_t* mask, int64_t n_gal, int32_t base_weight,
                                             int32_t n_parts, int64_t* starts_out) {
    if (!starts_out || base_weight < 0) {
        sps::set_last_error("sps_partition_galaxies: starts_out is NULL or base_weight < 0");
        return SPS_E_INVALID_ARG;
    }
    if (n_gal < 0 || n_parts < 1) {
        sps::set_last_error("sps_partition_galaxies: n_gal < 0 or n_parts < 1");
        return SPS_E_SHAPE;
    }
    std::vector<int64_t> w((size_t)n_gal);
    int64_t total = 0, wmax = 0;
    for (int64_t g = 0; g < n_gal; ++g) {
        w[(size_t)g] = (int64_t)base_weight + (mask ? popcount32(mask[g]) : 0);
        total += w[(size_t)g];
    }
    if (total == 0) {                     // nothing to weigh: balance the counts
        std::fill(w.begin(), w.end(), 1);
        total = n_gal;
    }
    for (int64_t x : w) wmax = std::max(wmax, x);
    int64_t lo = wmax, hi = std::max<int64_t>(total, 1);
    while (lo < hi) {                     // smallest T the greedy scan fits in n_parts blocks
        const int64_t mid = lo + (hi - lo) / 2;
        if (blocks_needed(w, mid) <= n_parts) hi = mid;
        else lo = mid + 1;
    }
    const int64_t T = lo;
    int64_t p = 0, cur = 0;
    starts_out[0] = 0;
    for (int64_t g = 0; g < n_gal; ++g) {
        const bool nonempty = g > starts_out[p];
        const bool must_cut = nonempty && (n_gal - g) <= (int64_t)n_parts - p - 1;
        if (nonempty && (must_cut || cur + w[(size_t)g] > T) && p + 1 < n_parts) {
            starts_out[++p] = g;
            cur = 0;
        }
        cur += w[(size_t)g];
    }
    for (int64_t q = p + 1; q <= n_parts; ++q) starts_out[q] = n_gal;
    return SPS_OK;
}
