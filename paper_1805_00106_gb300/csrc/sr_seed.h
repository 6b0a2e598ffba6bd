// sr_seed.h -- seed arithmetic shared by the host index (sr_index.cpp) and the
// device CAL finder (sr_cal.cu), so both derive bucket, key and orientation of a
// seed from one definition (Sec. 3.1: seeds, their reverse complements and the
// hashed address / key split of the pointer table).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define SR_HD __host__ __device__ __forceinline__
#else
#define SR_HD inline
#endif

namespace sr {

SR_HD uint64_t mask_bits(int bits) { return bits >= 64 ? ~0ull : ((1ull << bits) - 1ull); }

// invertible mix of the 2k-bit canonical seed (xor, odd multiplies, xor-shifts
// mod 2^(2k)): address + key identify the seed exactly (Sec. 3.1 hashing keeps
// the exact-match semantics of the key comparison).
SR_HD uint64_t seed_hash(uint64_t x, int k, uint64_t seed) {
  const int bits = 2 * k;
  const uint64_t M = mask_bits(bits);
  x = (x ^ seed) & M;
  x = (x * 0x9E3779B97F4A7C15ull) & M;
  x ^= x >> ((bits + 1) / 2);
  x = (x * 0xC2B2AE3D27D4EB4Full) & M;
  x ^= x >> ((bits + 2) / 3);
  return x & M;
}

// a k-mer and its reverse complement, 2 bits per base, first base highest
struct Kmer {
  uint64_t fwd = 0, rc = 0;
};

SR_HD void kmer_push(Kmer& km, uint8_t c, int k) {
  const uint64_t M = mask_bits(2 * k);
  km.fwd = ((km.fwd << 2) | c) & M;
  km.rc = (km.rc >> 2) | (static_cast<uint64_t>(3u - c) << (2 * (k - 1)));
}

}  // namespace sr
