// Oracle: Philox4x32-10 counter-based generator. TEST INFRASTRUCTURE ONLY.
//
// The paper (Sec. 2.C.3) rotates the directors "via a GPU-based pseudo-random
// number generator" without naming it.  Both paths use Philox4x32-10 as
// published by Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3" (SC'11): a 10-round Feistel-like bijection on four 32-bit
// words, each round multiplying words 0 and 2 by fixed odd constants and
// mixing the high halves with the other words and the key; the two-word key
// is bumped by the Weyl constants between rounds.
#include "internal.h"

namespace cgo {

void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kWeyl0;
      k1 += kWeyl1;
    }
    uint64_t p0 = (uint64_t)kMul0 * c0;
    uint64_t p1 = (uint64_t)kMul1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

}  // namespace cgo
