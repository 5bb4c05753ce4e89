// A user's program of the device API (include/wc_device_api.cuh): its own kernels insert,
// look up and erase single elements, and call for_each / for_all with device lambdas.
// Test infrastructure: built by tests/test_device_api_gpu.py, called through ctypes.
#include <cooperative_groups.h>
#include <cstdint>

#include "wc_device_api.cuh"

namespace {

// Keys of the fused producer: an odd-multiplier bijection of the index, so distinct.
__host__ __device__ uint32_t fused_key(uint64_t i, uint32_t seed) {
  return static_cast<uint32_t>(i * 2654435761ull) ^ seed;
}

template <class K>
__global__ void k_insert(wc_device_view v, const K* keys, const K* vals, uint64_t n, uint32_t* flags) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t f = wc_dev::insert<K>(v, keys[i], vals[i]);
    if (f) atomicOr(flags, f);
  }
}

// Grid-stride inserts that count their new keys per thread and add them to the size once.
template <class K>
__global__ void k_insert_uncounted(wc_device_view v, const K* keys, const K* vals, uint64_t n, uint32_t* flags) {
  long long added = 0;
  uint32_t f = 0;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t r = wc_dev::insert_uncounted<K>(v, keys[i], vals[i]);
    if (r == 0) ++added;
    f |= r;
  }
  wc_dev::add_size(v, added);
  if (f) atomicOr(flags, f);
}

template <class K>
__global__ void k_retrieve(wc_device_view v, const K* keys, uint64_t n, K* out, uint8_t* found) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    K x = K(~K(0));
    found[i] = wc_dev::retrieve<K>(v, keys[i], x) ? 1 : 0;
    out[i] = x;
  }
}

template <class K>
__global__ void k_erase(wc_device_view v, const K* keys, uint64_t n, unsigned long long* erased) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && wc_dev::erase<K>(v, keys[i])) atomicAdd(erased, 1ull);
}

// A fused pipeline: each thread produces its key and inserts it, no batch in memory.
__global__ void k_fused_insert(wc_device_view v, uint64_t n, uint32_t seed, uint32_t* flags) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t f = wc_dev::insert<uint32_t>(v, fused_key(i, seed), static_cast<uint32_t>(i));
    if (f) atomicOr(flags, f);
  }
}

// Per-element appends to a bucket multi-value table, all in one launch (concurrent).
// Grid-stride appends that count values and new keys per thread and add them once.
template <class K, class V>
__global__ void k_mv_append_uncounted(wc_device_view v, const K* keys, const V* vals, uint64_t n, uint32_t* flags) {
  wc_dev::bl::Counts c;
  uint32_t f = 0;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    f |= wc_dev::append_uncounted<K, V>(v, keys[i], vals[i], c);
  wc_dev::add_counts(v, c);
  if (f) atomicOr(flags, f);
}

template <class K, class V>
__global__ void k_mv_append(wc_device_view v, const K* keys, const V* vals, uint64_t n, uint32_t* flags) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t f = wc_dev::append<K, V>(v, keys[i], vals[i]);
    if (f) atomicOr(flags, f);
  }
}

// Hash sets: op 0 insert (out[i] = 1 if stored now), 1 contains, 2 erase (out[i] = 1 if erased).
template <class K>
__global__ void k_set_op(wc_device_view v, int op, const K* keys, uint64_t n, uint8_t* out, uint32_t* flags) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (op == 0) {
    const uint32_t f = wc_dev::set_insert<K>(v, keys[i]);
    if (f) atomicOr(flags, f);
    out[i] = f == 0 ? 1 : 0;
  } else if (op == 1) {
    out[i] = wc_dev::set_contains<K>(v, keys[i]) ? 1 : 0;
  } else {
    out[i] = wc_dev::set_erase<K>(v, keys[i]) ? 1 : 0;
  }
}

// Counting tables: add weights[i] (1 when weights is null) to keys[i]'s count; read counts.
template <class K>
__global__ void k_count_add(wc_device_view v, const K* keys, const K* weights, uint64_t n, uint32_t* flags) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t f = wc_dev::count_add<K>(v, keys[i], weights ? weights[i] : K(1));
    if (f) atomicOr(flags, f);
  }
}

template <class K>
__global__ void k_count_get(wc_device_view v, const K* keys, uint64_t n, K* out, uint8_t* found) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    K c = 0;
    found[i] = wc_dev::count_get<K>(v, keys[i], c) ? 1 : 0;
    out[i] = c;
  }
}

// Group-cooperative inserts and lookups: each tile of G threads serves one key.
template <class K, int W, int G>
__global__ void k_group_op(wc_device_view v, int op, const K* keys, const K* vals, uint64_t n, K* out, uint8_t* found,
                           uint32_t* flags) {
  namespace cg = cooperative_groups;
  const auto tile = cg::tiled_partition<G>(cg::this_thread_block());
  const uint64_t i = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / G;
  if (i >= n) return;  // whole tiles leave together (n is counted in tiles)
  if (op == 0) {
    const uint32_t f = wc_dev::insert_group<K, W, G>(tile, v, keys[i], vals[i]);
    if (f && tile.thread_rank() == 0) atomicOr(flags, f);
  } else {
    K x = K(~K(0));
    const bool hit = wc_dev::retrieve_group<K, W, G>(tile, v, keys[i], x);
    if (tile.thread_rank() == 0) {
      out[i] = hit ? x : K(~K(0));
      found[i] = hit ? 1 : 0;
    }
  }
}

template <class K, int W, int G>
int launch_group(const wc_device_view& v, int op, const void* keys, const void* vals, uint64_t n, void* out,
                 uint8_t* found, uint32_t* flags) {
  const uint64_t threads = n * G;
  k_group_op<K, W, G><<<static_cast<unsigned>((threads + 255) / 256), 256>>>(
      v, op, static_cast<const K*>(keys), static_cast<const K*>(vals), n, static_cast<K*>(out), found, flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

unsigned grid(uint64_t n) { return static_cast<unsigned>((n + 255) / 256); }

}  // namespace

extern "C" {

int wcu_insert(const wc_device_view* v, const void* keys, const void* vals, uint64_t n, uint32_t* flags) {
  if (n == 0) return 0;
  if (v->key_bytes == 4)
    k_insert<uint32_t><<<grid(n), 256>>>(*v, static_cast<const uint32_t*>(keys), static_cast<const uint32_t*>(vals), n,
                                        flags);
  else
    k_insert<unsigned long long><<<grid(n), 256>>>(*v, static_cast<const unsigned long long*>(keys),
                                                  static_cast<const unsigned long long*>(vals), n, flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_insert_uncounted(const wc_device_view* v, const void* keys, const void* vals, uint64_t n, uint32_t* flags) {
  if (n == 0) return 0;
  if (v->key_bytes == 4)
    k_insert_uncounted<uint32_t><<<64, 256>>>(*v, static_cast<const uint32_t*>(keys), static_cast<const uint32_t*>(vals),
                                             n, flags);
  else
    k_insert_uncounted<unsigned long long><<<64, 256>>>(*v, static_cast<const unsigned long long*>(keys),
                                                       static_cast<const unsigned long long*>(vals), n, flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_retrieve(const wc_device_view* v, const void* keys, uint64_t n, void* out, uint8_t* found) {
  if (n == 0) return 0;
  if (v->key_bytes == 4)
    k_retrieve<uint32_t><<<grid(n), 256>>>(*v, static_cast<const uint32_t*>(keys), n, static_cast<uint32_t*>(out),
                                          found);
  else
    k_retrieve<unsigned long long><<<grid(n), 256>>>(*v, static_cast<const unsigned long long*>(keys), n,
                                                    static_cast<unsigned long long*>(out), found);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_erase(const wc_device_view* v, const void* keys, uint64_t n, unsigned long long* erased) {
  if (n == 0) return 0;
  if (v->key_bytes == 4)
    k_erase<uint32_t><<<grid(n), 256>>>(*v, static_cast<const uint32_t*>(keys), n, erased);
  else
    k_erase<unsigned long long><<<grid(n), 256>>>(*v, static_cast<const unsigned long long*>(keys), n, erased);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_mv_append(const wc_device_view* v, const void* keys, const void* vals, uint64_t n, uint32_t* flags) {
  if (n == 0) return 0;
  if (v->key_bytes == 4 && v->value_bytes == 4)
    k_mv_append<uint32_t, uint32_t><<<grid(n), 256>>>(*v, static_cast<const uint32_t*>(keys),
                                                      static_cast<const uint32_t*>(vals), n, flags);
  else if (v->key_bytes == 8 && v->value_bytes == 4)
    k_mv_append<unsigned long long, uint32_t><<<grid(n), 256>>>(*v, static_cast<const unsigned long long*>(keys),
                                                                static_cast<const uint32_t*>(vals), n, flags);
  else if (v->key_bytes == 8)
    k_mv_append<unsigned long long, unsigned long long><<<grid(n), 256>>>(
        *v, static_cast<const unsigned long long*>(keys), static_cast<const unsigned long long*>(vals), n, flags);
  else
    k_mv_append<uint32_t, unsigned long long><<<grid(n), 256>>>(*v, static_cast<const uint32_t*>(keys),
                                                                static_cast<const unsigned long long*>(vals), n, flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_mv_append_uncounted(const wc_device_view* v, const void* keys, const void* vals, uint64_t n, uint32_t* flags) {
  if (n == 0) return 0;
  if (v->key_bytes == 4 && v->value_bytes == 4)
    k_mv_append_uncounted<uint32_t, uint32_t><<<128, 256>>>(*v, static_cast<const uint32_t*>(keys),
                                                           static_cast<const uint32_t*>(vals), n, flags);
  else if (v->key_bytes == 8 && v->value_bytes == 4)
    k_mv_append_uncounted<unsigned long long, uint32_t><<<128, 256>>>(
        *v, static_cast<const unsigned long long*>(keys), static_cast<const uint32_t*>(vals), n, flags);
  else if (v->key_bytes == 8)
    k_mv_append_uncounted<unsigned long long, unsigned long long><<<128, 256>>>(
        *v, static_cast<const unsigned long long*>(keys), static_cast<const unsigned long long*>(vals), n, flags);
  else
    k_mv_append_uncounted<uint32_t, unsigned long long><<<128, 256>>>(
        *v, static_cast<const uint32_t*>(keys), static_cast<const unsigned long long*>(vals), n, flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_set_op(const wc_device_view* v, int op, const void* keys, uint64_t n, uint8_t* out, uint32_t* flags) {
  if (n == 0) return 0;
  if (v->key_bytes == 4)
    k_set_op<uint32_t><<<grid(n), 256>>>(*v, op, static_cast<const uint32_t*>(keys), n, out, flags);
  else
    k_set_op<unsigned long long><<<grid(n), 256>>>(*v, op, static_cast<const unsigned long long*>(keys), n, out,
                                                  flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_count_add(const wc_device_view* v, const void* keys, const void* weights, uint64_t n, uint32_t* flags) {
  if (n == 0) return 0;
  if (v->key_bytes == 4)
    k_count_add<uint32_t><<<grid(n), 256>>>(*v, static_cast<const uint32_t*>(keys),
                                           static_cast<const uint32_t*>(weights), n, flags);
  else
    k_count_add<unsigned long long><<<grid(n), 256>>>(*v, static_cast<const unsigned long long*>(keys),
                                                     static_cast<const unsigned long long*>(weights), n, flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

int wcu_count_get(const wc_device_view* v, const void* keys, uint64_t n, void* out, uint8_t* found) {
  if (n == 0) return 0;
  if (v->key_bytes == 4)
    k_count_get<uint32_t><<<grid(n), 256>>>(*v, static_cast<const uint32_t*>(keys), n, static_cast<uint32_t*>(out),
                                           found);
  else
    k_count_get<unsigned long long><<<grid(n), 256>>>(*v, static_cast<const unsigned long long*>(keys), n,
                                                     static_cast<unsigned long long*>(out), found);
  return static_cast<int>(cudaDeviceSynchronize());
}

// Group-cooperative op (0 insert, 1 lookup) with tiles of G threads; (key width, W, G) as
// the tests use them.
int wcu_group_op(const wc_device_view* v, int op, int G, const void* keys, const void* vals, uint64_t n, void* out,
                 uint8_t* found, uint32_t* flags) {
  if (n == 0) return 0;
  const int W = static_cast<int>(v->window_width);
#define WCU_G(K, Wv, Gv) \
  if (W == (Wv) && G == (Gv)) return launch_group<K, Wv, Gv>(*v, op, keys, vals, n, out, found, flags);
  if (v->key_bytes == 4) {
    WCU_G(uint32_t, 8, 1) WCU_G(uint32_t, 8, 2) WCU_G(uint32_t, 8, 4) WCU_G(uint32_t, 16, 4) WCU_G(uint32_t, 32, 8)
  } else {
    WCU_G(unsigned long long, 4, 2) WCU_G(unsigned long long, 8, 4) WCU_G(unsigned long long, 2, 2)
  }
#undef WCU_G
  return -1;
}

// Write one 8-byte word of device memory from the host (the tests' way to leave a list
// handle blocked, as if its owner had stopped).
int wcu_poke_u64(void* dptr, uint64_t value) {
  return static_cast<int>(cudaMemcpy(dptr, &value, 8, cudaMemcpyHostToDevice));
}

int wcu_fused_insert(const wc_device_view* v, uint64_t n, uint32_t seed, uint32_t* flags) {
  if (n == 0) return 0;
  k_fused_insert<<<grid(n), 256>>>(*v, n, seed, flags);
  return static_cast<int>(cudaDeviceSynchronize());
}

// for_each: sum and count of the values found, and the found mask.
int wcu_for_each(const wc_device_view* v, const void* keys, uint64_t n, unsigned long long* sums, uint8_t* found) {
  cudaError_t e;
  if (v->key_bytes == 4) {
    e = wc_dev::for_each(*v, static_cast<const uint32_t*>(keys), n,
                         [sums, found] __device__(uint32_t, uint32_t val, uint64_t i) {
                           atomicAdd(sums, static_cast<unsigned long long>(val));
                           atomicAdd(sums + 1, 1ull);
                           found[i] = 1;
                         });
  } else {
    e = wc_dev::for_each(*v, static_cast<const unsigned long long*>(keys), n,
                         [sums, found] __device__(unsigned long long, unsigned long long val, uint64_t i) {
                           atomicAdd(sums, val);
                           atomicAdd(sums + 1, 1ull);
                           found[i] = 1;
                         });
  }
  if (e != cudaSuccess) return static_cast<int>(e);
  return static_cast<int>(cudaDeviceSynchronize());
}

// for_all: number of stored pairs, sum of their keys and of their values.
int wcu_for_all(const wc_device_view* v, unsigned long long* sums) {
  cudaError_t e;
  if (v->key_bytes == 4) {
    e = wc_dev::for_all<uint32_t>(*v, [sums] __device__(uint32_t k, uint32_t val, uint64_t) {
      atomicAdd(sums, 1ull);
      atomicAdd(sums + 1, static_cast<unsigned long long>(k));
      atomicAdd(sums + 2, static_cast<unsigned long long>(val));
    });
  } else {
    e = wc_dev::for_all<unsigned long long>(*v, [sums] __device__(unsigned long long k, unsigned long long val,
                                                                   uint64_t) {
      atomicAdd(sums, 1ull);
      atomicAdd(sums + 1, k);
      atomicAdd(sums + 2, val);
    });
  }
  if (e != cudaSuccess) return static_cast<int>(e);
  return static_cast<int>(cudaDeviceSynchronize());
}

}  // extern "C"
