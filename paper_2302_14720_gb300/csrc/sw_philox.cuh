// sw_philox.cuh -- device-side Philox-4x32-10 for libsw (conventions C4-C7
// of include/sw.h).
//
// Philox-4x32 is the counter-based generator of Salmon, Moraes, Dror and
// Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): each of ten
// rounds multiplies words 0 and 2 by two fixed 32-bit constants, xors the
// high halves of the products with the other two words and the round key,
// and permutes the words; the key advances by two Weyl increments between
// rounds. The key schedule is uniform across a launch, so the host expands it
// once into a KeySchedule kernel parameter and the rounds read it from the
// constant bank instead of adding the increments per call.
#pragma once
#include <stdint.h>

namespace sw {

constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

struct KeySchedule {
  uint32_t k0[10];
  uint32_t k1[10];
};

// Host and device: round keys of the 10 rounds for a 64-bit seed
// (key = (seed low word, seed high word)).
__host__ __device__ inline KeySchedule make_key_schedule(uint64_t seed) {
  KeySchedule ks;
  uint32_t a = (uint32_t)(seed & 0xffffffffu), b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    ks.k0[r] = a;
    ks.k1[r] = b;
    a += kPhiloxWeylA;
    b += kPhiloxWeylB;
  }
  return ks;
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, const KeySchedule& ks) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa = (uint64_t)kPhiloxMulA * c.x;
    const uint64_t pb = (uint64_t)kPhiloxMulB * c.z;
    c = make_uint4((uint32_t)(pb >> 32) ^ c.y ^ ks.k0[r], (uint32_t)pb,
                   (uint32_t)(pa >> 32) ^ c.w ^ ks.k1[r], (uint32_t)pa);
  }
  return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4& q, uint32_t j) {
  return j == 0u ? q.x : j == 1u ? q.y : j == 2u ? q.z : q.w;
}

// C6: site index i owns bit (i & 31) of word (i >> 5) & 3 of block
// (i >> 7, t, 1, 0); the cluster rooted at `root` flips in sweep t iff the
// bit of index root is set.
__device__ __forceinline__ uint32_t flip_bit(uint32_t root, uint32_t t, const KeySchedule& ks) {
  const uint4 q = philox4x32_10(make_uint4(root >> 7, t, 1u, 0u), ks);
  return (word_of(q, (root >> 5) & 3u) >> (root & 31u)) & 1u;
}

// The C6 bits of the 32 consecutive indices i0 .. i0+31 (bit k for i0 + k):
// one block when i0 is a multiple of 32, else the two 32-bit words that the
// range straddles (a second block only when they lie in different blocks).
__device__ __forceinline__ uint32_t flip_bits32(uint32_t i0, uint32_t t, const KeySchedule& ks) {
  const uint32_t a = i0 >> 5, o = i0 & 31u, j = a & 3u;
  const uint4 q = philox4x32_10(make_uint4(a >> 2, t, 1u, 0u), ks);
  const uint32_t lo = word_of(q, j);
  if (o == 0u) return lo;
  const uint32_t hi = j < 3u ? word_of(q, j + 1u) : philox4x32_10(make_uint4((a >> 2) + 1u, t, 1u, 0u), ks).x;
  return (lo >> o) | (hi << (32u - o));
}

// §2.4 as printed (the assignment rule): the cluster rooted at `root` gets
// spin -1 in sweep t iff the top bit of word x0 of block (root, t, 3, 0) is set.
__device__ __forceinline__ uint32_t assign_bit(uint32_t root, uint32_t t, const KeySchedule& ks) {
  return philox4x32_10(make_uint4(root, t, 3u, 0u), ks).x >> 31;
}

// The per-cluster decision of a sweep: the flip bit (rule 0) or the new
// spin's sign bit (rule 1). A site's new sign bit is decision ^ (rule 0 ?
// its old sign bit : 0).
__device__ __forceinline__ uint32_t decision_bit(uint32_t root, uint32_t t, const KeySchedule& ks, uint32_t rule) {
  return rule ? assign_bit(root, t, ks) : flip_bit(root, t, ks);
}

// §6 (q-state Potts): the cluster rooted at `root` takes state
// floor(x0 q / 2^32) in sweep t, x0 the first word of block (root, t, 3, 0);
// for q = 2 this is the assignment rule's sign bit.
__device__ __forceinline__ uint32_t potts_new_state(uint32_t root, uint32_t t, const KeySchedule& ks, uint32_t q) {
  return (uint32_t)(((uint64_t)philox4x32_10(make_uint4(root, t, 3u, 0u), ks).x * q) >> 32);
}

}  // namespace sw
