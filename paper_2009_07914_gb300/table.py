"""Object wrappers over the C-ABI functions: a table owns its handle, and the methods
allocate outputs on the table's device.  Inputs may be CUDA tensors or numpy arrays
(numpy arrays are copied to the device first)."""
from __future__ import annotations

import numpy as np
import torch

from . import api
from ._binding import WC_BLOOM_FILTER, WC_COUNTING, WC_HASH_SET, WC_MULTI_VALUE, WC_MULTI_VALUE_OA, WC_SINGLE_VALUE

_INT = {4: torch.int32, 8: torch.int64}
_NP_SIGNED = {4: np.int32, 8: np.int64}
_NP_UNSIGNED = {4: np.uint32, 8: np.uint64}


def to_device(a, width: int, device) -> torch.Tensor:
    """Bit-copy of an integer array onto the device as a signed tensor of `width` bytes."""
    if isinstance(a, torch.Tensor):
        if a.element_size() != width:
            raise ValueError("element width %d, expected %d" % (a.element_size(), width))
        return a.to(device).contiguous()
    arr = np.ascontiguousarray(np.asarray(a).astype(_NP_UNSIGNED[width], copy=False))
    return torch.from_numpy(arr.view(_NP_SIGNED[width])).to(device)


def to_numpy(t: torch.Tensor, width: int) -> np.ndarray:
    return t.cpu().numpy().view(_NP_UNSIGNED[width])


class _Table:
    kind = -1

    def __init__(self, key_bytes=4, value_bytes=4, min_capacity=1024, window_width=0, value_pool_capacity=0,
                 seed=0x5EED_C0DE, device=None, l2_persist=False, options=0, bucket_first_size=0, bucket_growth=1.0):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.kb, self.vb = key_bytes, value_bytes
        self.handle = api.wc_table_create(self.kind, key_bytes, value_bytes, min_capacity, window_width,
                                          value_pool_capacity, seed, self.device.index, l2_persist, options,
                                          bucket_first_size, bucket_growth)
        self.info = api.wc_table_get_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize(self.device)
            api.wc_table_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def capacity(self) -> int:
        return self.info["capacity"]

    def keys_dev(self, keys) -> torch.Tensor:
        return to_device(keys, self.kb, self.device)

    def values_dev(self, values) -> torch.Tensor:
        return to_device(values, self.vb, self.device)

    def insert(self, keys, values, stream=None):
        k, v = self.keys_dev(keys), self.values_dev(values)
        api.wc_insert(self.handle, k, v, stream=stream)
        return api.wc_get_status(self.handle, clear=True, stream=stream)

    def erase(self, keys, stream=None):
        api.wc_erase(self.handle, self.keys_dev(keys), stream=stream)
        return api.wc_get_status(self.handle, clear=True, stream=stream)

    def clear(self, stream=None):
        api.wc_table_clear(self.handle, stream)

    def size(self, stream=None) -> int:
        return api.wc_size(self.handle, stream)

    def num_keys(self, stream=None) -> int:
        return api.wc_num_keys(self.handle, stream)

    def load_factor(self, stream=None) -> float:
        return api.wc_load_factor(self.handle, stream)

    def status(self, clear=False, stream=None) -> int:
        return api.wc_get_status(self.handle, clear, stream)

    def set_launch(self, op, group_size, block_threads=256, blocks_per_sm=0, scheme=0, region_mib=0,
                   keys_in_flight=0):
        api.wc_table_set_launch(self.handle, op, group_size, block_threads, blocks_per_sm, scheme, region_mib,
                                keys_in_flight)


class SingleValueTable(_Table):
    kind = WC_SINGLE_VALUE

    def retrieve(self, keys, stream=None):
        """Returns (values, found, flags) as numpy arrays (values as unsigned)."""
        k = self.keys_dev(keys)
        out = torch.empty(k.numel(), dtype=_INT[self.vb], device=self.device)
        found = torch.empty(k.numel(), dtype=torch.uint8, device=self.device)
        api.wc_retrieve(self.handle, k, out, found, stream=stream)
        flags = api.wc_get_status(self.handle, clear=True, stream=stream)
        return to_numpy(out, self.vb), found.cpu().numpy(), flags


class MultiValueTable(_Table):
    kind = WC_MULTI_VALUE

    def pool_used(self, stream=None) -> int:
        return api.wc_value_pool_used(self.handle, stream)

    def count_values(self, keys, stream=None):
        k = self.keys_dev(keys)
        offs = torch.empty(k.numel() + 1, dtype=torch.int64, device=self.device)
        api.wc_count_values(self.handle, k, offs, stream=stream)
        flags = api.wc_get_status(self.handle, clear=True, stream=stream)
        return to_numpy(offs, 8), flags

    def retrieve_multi(self, keys, offsets, stream=None):
        k = self.keys_dev(keys)
        offs = to_device(offsets, 8, self.device)
        total = int(np.asarray(offsets)[-1]) if not isinstance(offsets, torch.Tensor) else int(offsets[-1])
        out = torch.empty(max(total, 1), dtype=_INT[self.vb], device=self.device)
        api.wc_retrieve_multi(self.handle, k, offs, out, stream=stream)
        flags = api.wc_get_status(self.handle, clear=True, stream=stream)
        return to_numpy(out, self.vb)[:total], flags


class MultiValueOATable(MultiValueTable):
    """Open-addressing multi-value table: one slot per stored pair (4+4 or 8+8 bytes)."""
    kind = WC_MULTI_VALUE_OA


class CountingTable(SingleValueTable):
    """Occurrence counts per key (key and count of the same width, 4 or 8 bytes)."""
    kind = WC_COUNTING

    def __init__(self, key_bytes=4, min_capacity=1024, **kw):
        super().__init__(key_bytes, key_bytes, min_capacity=min_capacity, **kw)

    def insert(self, keys, weights=None, stream=None):
        k = self.keys_dev(keys)
        w = None if weights is None else self.values_dev(weights)
        api.wc_insert(self.handle, k, w, stream=stream)
        return api.wc_get_status(self.handle, clear=True, stream=stream)


class _Membership(_Table):
    def insert(self, keys, stream=None):
        api.wc_insert(self.handle, self.keys_dev(keys), None, stream=stream)
        return api.wc_get_status(self.handle, clear=True, stream=stream)

    def contains(self, keys, stream=None):
        """Returns (found mask as numpy uint8, flags)."""
        k = self.keys_dev(keys)
        found = torch.empty(k.numel(), dtype=torch.uint8, device=self.device)
        api.wc_contains(self.handle, k, found, stream=stream)
        return found.cpu().numpy(), api.wc_get_status(self.handle, clear=True, stream=stream)


class HashSetTable(_Membership):
    """A set of 4- or 8-byte keys, one key per slot."""
    kind = WC_HASH_SET

    def __init__(self, key_bytes=4, min_capacity=1024, **kw):
        super().__init__(key_bytes, 0, min_capacity=min_capacity, **kw)


class BloomFilterTable(_Membership):
    """Blocked Bloom filter of `bits` bits (whole 256-bit blocks), k bits per key."""
    kind = WC_BLOOM_FILTER

    def __init__(self, key_bytes=4, bits=1 << 20, k=8, seed=0x5EED_C0DE, device=None):
        super().__init__(key_bytes, 0, min_capacity=bits, window_width=k, seed=seed, device=device)
