// bwt_inverse_check: host inverse of one block by the LF walk.
//
// Section 3.1 of the paper notes that the inverse transform can start from
// any row of the output. Here one walk starts at the primary row: row r
// holds rotation SA[r] and L[r] = S[SA[r] - 1], and the LF mapping
// LF(r) = C[L[r]] + (count of L[r] in L[0..r-1]) (C[c] = bytes smaller than
// c) gives the row of rotation SA[r] - 1, so the walk emits S back to front.
#include <cstdint>
#include <cstring>
#include <vector>

#include "bwt.h"

extern "C" bwt_status bwt_inverse_check(const uint8_t* L, uint64_t n, int32_t primary, const uint8_t* original) {
    if (!L || !original || n == 0 || primary < 0 || (uint64_t)primary >= n) return BWT_EINVAL;
    uint64_t count[256];
    std::memset(count, 0, sizeof(count));
    uint64_t ref[256];
    std::memset(ref, 0, sizeof(ref));
    for (uint64_t k = 0; k < n; ++k) {
        ++count[L[k]];
        ++ref[original[k]];
    }
    if (std::memcmp(count, ref, sizeof(count)) != 0) return BWT_EMISMATCH;  // L is not a permutation of S
    uint64_t first[256];
    uint64_t acc = 0;
    for (int c = 0; c < 256; ++c) {
        first[c] = acc;
        acc += count[c];
    }
    std::vector<uint64_t> lf(n);
    uint64_t seen[256];
    std::memset(seen, 0, sizeof(seen));
    for (uint64_t k = 0; k < n; ++k) lf[k] = first[L[k]] + seen[L[k]]++;
    uint64_t r = (uint64_t)primary;
    for (uint64_t i = n; i-- > 0;) {
        if (L[r] != original[i]) return BWT_EMISMATCH;
        r = lf[r];
    }
    return BWT_OK;
}
