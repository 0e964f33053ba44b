// Tile geometry shared by the apply kernels (host code).
//
// A CTA owns a tile of 2^TB amplitudes: the index bits [0, L) plus the h targets at or
// above L, with L + h = TB.  The tile is 2^h contiguous segments of 2^L amplitudes.
#pragma once

#include <cstdint>

#include "sv.h"

namespace svk {

struct Plan {
    uint32_t L = 0, h = 0;
    uint32_t hi[SV_MAX_K] = {0, 0, 0, 0, 0};
    uint32_t lp[SV_MAX_K] = {0, 0, 0, 0, 0};
    unsigned long long ntiles = 1;
};

// Largest L with L + #{targets >= L} <= TB (then equality holds); whole state if small.
inline Plan make_plan(uint32_t n, uint32_t k, const uint32_t *t, uint32_t TB) {
    Plan p;
    if (n <= TB) {
        p.L = n;
        p.h = 0;
    } else {
        for (uint32_t L = TB;; --L) {
            uint32_t h = 0;
            for (uint32_t j = 0; j < k; ++j) h += t[j] >= L;
            if (L + h <= TB) {
                p.L = L;
                p.h = h;
                break;
            }
        }
    }
    uint32_t nh = 0;
    for (uint32_t j = 0; j < k; ++j) {
        if (t[j] >= p.L) {
            p.lp[j] = p.L + nh;
            p.hi[nh++] = t[j];
        } else {
            p.lp[j] = t[j];
        }
    }
    p.ntiles = 1ull << (n - p.L - p.h);
    return p;
}

}  // namespace svk
