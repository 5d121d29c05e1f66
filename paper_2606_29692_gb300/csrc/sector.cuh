// Rank of a qubit-space basis index in a sector (fixed alpha and beta
// electron counts), or -1 outside it.  Decodes the occupation bits with the
// rows of B^-1 (JW: the index itself), then ranks the occupied alpha and
// beta spatial orbitals colexicographically: sum_j C(c_j, j).
#pragma once

#include "dev.cuh"

namespace tq {

__device__ __forceinline__ long long sector_rank(uint32_t e, const SectorSpec& s) {
    uint32_t occ = e;
    if (s.mapping != TQ_JW) {
        occ = 0;
        for (int j = 0; j < s.nq; ++j) occ |= (uint32_t)parity32(e & s.dec[j]) << j;
    }
    int ja = 0, jb = 0;
    long long ra = 0, rb = 0;
    for (int p = 0; p < s.n; ++p) {
        if ((occ >> (2 * p)) & 1u) {
            ++ja;
            if (ja <= s.na) ra += s.binom[p][ja];
        }
        if ((occ >> (2 * p + 1)) & 1u) {
            ++jb;
            if (jb <= s.nb) rb += s.binom[p][jb];
        }
    }
    if (ja != s.na || jb != s.nb) return -1;
    return ra * s.binom[s.n][s.nb] + rb;
}

}  // namespace tq
