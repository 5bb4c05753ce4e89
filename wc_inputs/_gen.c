/* Fast fills of the seeded streams defined in wc_inputs/__init__.py (same outputs as the
 * numpy definitions there; a test compares them).  Plain C, no method arithmetic. */
#include <stdint.h>

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* outputs start..start+count-1 of the SplitMix64 stream of `seed` */
void wcgen_splitmix64(uint64_t seed, uint64_t start, uint64_t count, uint64_t* out) {
  for (uint64_t i = 0; i < count; ++i) out[i] = sm64_mix(seed + (start + i + 1) * 0x9E3779B97F4A7C15ull);
}

/* high 32 bits of the stream (uniform uint32) */
void wcgen_splitmix64_hi32(uint64_t seed, uint64_t start, uint64_t count, uint32_t* out) {
  for (uint64_t i = 0; i < count; ++i)
    out[i] = (uint32_t)(sm64_mix(seed + (start + i + 1) * 0x9E3779B97F4A7C15ull) >> 32);
}

/* lowbias32 of the Weyl sequence base + i * 0x9E3779B9 (mod 2^32), i = start.. */
void wcgen_lowbias32_weyl(uint32_t base, uint64_t start, uint64_t count, uint32_t* out) {
  for (uint64_t i = 0; i < count; ++i) {
    uint32_t x = base + (uint32_t)(start + i) * 0x9E3779B9u;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    out[i] = x;
  }
}
