// Bloom filters (the paper's BloomFilter: set membership with false positives), blocked
// for the GPU: a key owns one 256-bit block (32 bytes, one sector) chosen by its hash and
// sets k bits inside it, so an insert is at most k atomic ORs into one sector and a lookup
// is one 32-byte read.
//   h = fmix64(key ^ seed); block = floor(hi32(h) * blocks / 2^32);
//   bit positions: bytes 0..7 of g1 = fmix64(h ^ 0x9e3779b97f4a7c15), then bytes of
//   g2 = fmix64(g1), ... (position i = byte i % 8 of g_{i / 8 + 1}); bits may coincide.
#include <cuda_runtime.h>

#include <cstdint>

#include "wc.h"
#include "wc_device.cuh"
#include "wc_internal.h"
#include "wc_launch.cuh"

namespace wc {
namespace {

// The key's block and its 8-word bit mask.
__device__ __forceinline__ uint64_t bloom_mask(uint64_t key, uint64_t seed, uint32_t blocks, int k, uint32_t (&m)[8]) {
  const uint64_t h = fmix64(key ^ seed);
  const uint64_t block = (static_cast<uint64_t>(static_cast<uint32_t>(h >> 32)) * blocks) >> 32;
#pragma unroll
  for (int i = 0; i < 8; ++i) m[i] = 0;
  uint64_t g = h ^ 0x9e3779b97f4a7c15ull;
  for (int i = 0; i < k; ++i) {
    if ((i & 7) == 0) g = fmix64(g);
    const uint32_t pos = static_cast<uint32_t>(g >> (8 * (i & 7))) & 255u;
#pragma unroll
    for (int wv = 0; wv < 8; ++wv)
      if ((pos >> 5) == static_cast<uint32_t>(wv)) m[wv] |= 1u << (pos & 31u);
  }
  return block;
}

template <class K>
__global__ void __launch_bounds__(256) k_bloom_insert(TableDesc t, const K* __restrict__ keys, uint64_t n, int k) {
  uint32_t* bits = static_cast<uint32_t*>(t.slots);
  uint32_t flags = 0;
  long long added = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const K key = ldg_stream(keys + i);
    if (key == K(0) || key == K(~K(0))) {
      flags |= kFlagInvalid;
      continue;
    }
    uint32_t m[8];
    const uint64_t b = bloom_mask(static_cast<uint64_t>(key), t.seed, t.p, k, m);
#pragma unroll
    for (int wv = 0; wv < 8; ++wv)
      if (m[wv]) atomicOr(bits + b * 8 + wv, m[wv]);
    ++added;
  }
  flush_flags(t.status, flags);
  flush_delta(t.size, added);
}

template <class K>
__global__ void __launch_bounds__(256) k_bloom_contains(TableDesc t, const K* __restrict__ keys, uint64_t n, int k,
                                                        uint8_t* __restrict__ found) {
  const unsigned long long* bits = static_cast<const unsigned long long*>(t.slots);
  uint32_t flags = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const K key = ldg_stream(keys + i);
    if (key == K(0) || key == K(~K(0))) {
      flags |= kFlagInvalid;
      found[i] = 0;
      continue;
    }
    uint32_t m[8];
    const uint64_t b = bloom_mask(static_cast<uint64_t>(key), t.seed, t.p, k, m);
    unsigned long long u[4];
    ldcg4(bits + b * 4, u);
    bool all = true;
#pragma unroll
    for (int wv = 0; wv < 4; ++wv) {
      const uint32_t lo = static_cast<uint32_t>(u[wv]), hi = static_cast<uint32_t>(u[wv] >> 32);
      all &= (lo & m[2 * wv]) == m[2 * wv] && (hi & m[2 * wv + 1]) == m[2 * wv + 1];
    }
    found[i] = all ? 1 : 0;
  }
  flush_flags(t.status, flags);
}

template <class K>
cudaError_t run(const wc_table* t, int op, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s) {
  const int k = t->cfg.window_width;
  const K* kk = static_cast<const K*>(keys);
  if (op == WC_OP_INSERT) {
    auto kern = k_bloom_insert<K>;
    const uint64_t want = (n + 255) / 256, most = static_cast<uint64_t>(occupancy(kern, 256)) * t->sm_count;
    return launch_k(t, kern, static_cast<unsigned>(want < most ? want : most), 256u, 0, s, desc_of(t), kk, n, k);
  }
  auto kern = k_bloom_contains<K>;
  const uint64_t want = (n + 255) / 256, most = static_cast<uint64_t>(occupancy(kern, 256)) * t->sm_count;
  return launch_k(t, kern, static_cast<unsigned>(want < most ? want : most), 256u, 0, s, desc_of(t), kk, n, k, found);
}

}  // namespace

// op: WC_OP_INSERT (set the keys' bits) or WC_OP_RETRIEVE (membership into found).
cudaError_t bloom_launch(const wc_table* t, int op, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s) {
  return t->cfg.key_bytes == 4 ? run<uint32_t>(t, op, keys, n, found, s) : run<unsigned long long>(t, op, keys, n, found, s);
}

}  // namespace wc
