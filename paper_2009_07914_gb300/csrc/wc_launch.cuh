// Grid sizing and launch helpers shared by the kernel families.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "wc_internal.h"

namespace wc {

// Resident blocks per SM of a kernel at `block` threads and `smem` dynamic shared bytes,
// cached by (kernel address, block, smem).
int occupancy_cached(const void* kernel, int block, size_t smem);

template <class Kernel>
int occupancy(Kernel kernel, int block) {
  return occupancy_cached(reinterpret_cast<const void*>(kernel), block, 0);
}

template <class Kernel>
int occupancy_smem(Kernel kernel, int block, size_t smem) {
  return occupancy_cached(reinterpret_cast<const void*>(kernel), block, smem);
}

// Persistent-style grid for the probe engines: at most blocks_per_sm * SMs blocks, and
// no more warps than one key per group needs; each warp owns `per_warp` consecutive
// input positions.
struct EngineGrid {
  unsigned blocks;
  uint64_t per_warp;
};

inline EngineGrid engine_grid(uint64_t n, int group, int block, int blocks_per_sm, int sms) {
  const uint64_t gpw = 32 / group;
  const uint64_t wpb = block / 32;
  const uint64_t want_warps = (n + gpw - 1) / gpw;
  const uint64_t want_blocks = std::max<uint64_t>(1, (want_warps + wpb - 1) / wpb);
  const uint64_t max_blocks = static_cast<uint64_t>(std::max(1, blocks_per_sm)) * std::max(1, sms);
  const uint64_t blocks = std::min(want_blocks, max_blocks);
  const uint64_t warps = blocks * wpb;
  return EngineGrid{static_cast<unsigned>(blocks), (n + warps - 1) / warps};
}

// cudaLaunchKernelEx with the table's L2 access-policy window, if it has one.
template <class... KArgs, class... Args>
cudaError_t launch_k(const wc_table* t, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                     cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  unsigned na = 0;
  cfg.attrs = l2_attr(t, attr, &na);
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace wc
