"""GB300-native forward Burrows-Wheeler block sort.

The transform (the paper's Section 3.1: sort the rotations of the block)
runs in hand-written sm_103a CUDA behind the C ABI of ``include/bwt.h``;
this package is the thin Python binding with the same names. PyTorch tensors
supply device memory and streams only.

    plan = Plan(max_blocks=64, max_total_bytes=64 * 900_000, max_block_bytes=900_000)
    L, primary = plan.forward(d_bytes, offsets)     # d_bytes: uint8 CUDA tensor
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (BWT_OK, BWTError, F_GRAPH, F_LEARNED, F_PER_BLOCK_LAUNCH, F_TIMING, PlanDesc, Stats,
                   check)

__all__ = ["Plan", "BWTError", "bwt_inverse_check", "F_GRAPH", "F_LEARNED", "F_PER_BLOCK_LAUNCH", "F_TIMING"]


def _ptr(t) -> int:
    return int(t.data_ptr())


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """bwt_plan_create / bwt_forward_batch / bwt_plan_destroy."""

    def __init__(self, max_blocks: int, max_total_bytes: int, max_block_bytes: int, radix_bits: int = 0,
                 tile_keys: int = 0, flags: int = 0, model_path: str | None = None, device: int = 0):
        self.lib = _lib.load()
        self.desc = PlanDesc(max_blocks, max_total_bytes, max_block_bytes, radix_bits, tile_keys, flags,
                             model_path.encode() if model_path else None)
        h = ctypes.c_void_p()
        check(self.lib.bwt_plan_create(ctypes.byref(self.desc), device, ctypes.byref(h)), "bwt_plan_create")
        self.handle = h
        self.device = device
        self.flags = flags

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.lib.bwt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def forward_into(self, d_in, offsets, d_L, d_primary, stream=None, raise_on_error: bool = True) -> int:
        """bwt_forward_batch on caller-owned buffers. `offsets` is a uint64 numpy
        array, a CPU tensor or a CUDA tensor with num_blocks + 1 entries."""
        if isinstance(offsets, np.ndarray):
            off = np.ascontiguousarray(offsets, dtype=np.uint64)
            off_ptr, nb = off.ctypes.data, off.size - 1
        else:
            off_ptr, nb = _ptr(offsets), offsets.numel() - 1
        st = self.lib.bwt_forward_batch(self.handle, _ptr(d_in), off_ptr, nb, _ptr(d_L), _ptr(d_primary),
                                        _stream_handle(stream))
        if raise_on_error:
            check(st, "bwt_forward_batch")
        return st

    def forward(self, d_in, offsets, stream=None):
        """Returns (L uint8 CUDA tensor, primary int32 CUDA tensor)."""
        import torch
        nb = (offsets.size if isinstance(offsets, np.ndarray) else offsets.numel()) - 1
        L = torch.empty_like(d_in)
        prim = torch.empty(nb, dtype=torch.int32, device=d_in.device)
        self.forward_into(d_in, offsets, L, prim, stream)
        return L, prim

    def inverse_into(self, d_L, offsets, d_primary, d_out, stream=None, raise_on_error: bool = True) -> int:
        """bwt_inverse_batch on caller-owned buffers (offsets as for forward_into)."""
        if isinstance(offsets, np.ndarray):
            off = np.ascontiguousarray(offsets, dtype=np.uint64)
            off_ptr, nb = off.ctypes.data, off.size - 1
        else:
            off_ptr, nb = _ptr(offsets), offsets.numel() - 1
        st = self.lib.bwt_inverse_batch(self.handle, _ptr(d_L), off_ptr, nb, _ptr(d_primary), _ptr(d_out),
                                        _stream_handle(stream))
        if raise_on_error:
            check(st, "bwt_inverse_batch")
        return st

    def inverse(self, d_L, offsets, d_primary, stream=None):
        """Returns the blocks (uint8 CUDA tensor) whose BWT is (d_L, d_primary)."""
        import torch
        out = torch.empty_like(d_L)
        self.inverse_into(d_L, offsets, d_primary, out, stream)
        return out

    @staticmethod
    def _offsets(offsets):
        if isinstance(offsets, np.ndarray):
            off = np.ascontiguousarray(offsets, dtype=np.uint64)
            return off, off.ctypes.data, off.size - 1
        return offsets, _ptr(offsets), offsets.numel() - 1

    def rle_encode_into(self, d_in, offsets, d_chars, d_lens, d_run_off, stream=None, raise_on_error=True) -> int:
        """bwt_rle_encode on caller-owned buffers (d_chars, d_lens sized like d_in)."""
        keep, off_ptr, nb = self._offsets(offsets)
        st = self.lib.bwt_rle_encode(self.handle, _ptr(d_in), off_ptr, nb, _ptr(d_chars), _ptr(d_lens),
                                     _ptr(d_run_off), _stream_handle(stream))
        if raise_on_error:
            check(st, "bwt_rle_encode")
        return st

    def rle_encode(self, d_in, offsets, stream=None):
        """(chars uint8, lens int32 (uint32 values), run_off int64 (uint64 values)) CUDA tensors,
        trimmed to the number of runs."""
        import torch
        nb = (offsets.size if isinstance(offsets, np.ndarray) else offsets.numel()) - 1
        chars = torch.empty_like(d_in)
        lens = torch.empty(d_in.numel(), dtype=torch.int32, device=d_in.device)
        run_off = torch.empty(nb + 1, dtype=torch.int64, device=d_in.device)
        self.rle_encode_into(d_in, offsets, chars, lens, run_off, stream)
        R = int(run_off[nb].item())
        return chars[:R], lens[:R], run_off

    def rle_decode_into(self, d_chars, d_lens, d_run_off, offsets, d_out, stream=None, raise_on_error=True) -> int:
        keep, off_ptr, nb = self._offsets(offsets)
        st = self.lib.bwt_rle_decode(self.handle, _ptr(d_chars), _ptr(d_lens), _ptr(d_run_off), off_ptr, nb,
                                     _ptr(d_out), _stream_handle(stream))
        if raise_on_error:
            check(st, "bwt_rle_decode")
        return st

    def rle_decode(self, d_chars, d_lens, d_run_off, offsets, stream=None):
        import torch
        total = int(offsets[-1]) if isinstance(offsets, np.ndarray) else int(offsets[-1].item())
        out = torch.empty(total, dtype=torch.uint8, device=d_chars.device)
        self.rle_decode_into(d_chars, d_lens, d_run_off, offsets, out, stream)
        return out

    def vle_encode_into(self, d_in, offsets, d_code, d_len, d_out, d_byte_off, d_block_bits, stream=None,
                        raise_on_error=True) -> int:
        keep, off_ptr, nb = self._offsets(offsets)
        st = self.lib.bwt_vle_encode(self.handle, _ptr(d_in), off_ptr, nb, _ptr(d_code), _ptr(d_len), _ptr(d_out),
                                     d_out.numel(), _ptr(d_byte_off), _ptr(d_block_bits), _stream_handle(stream))
        if raise_on_error:
            check(st, "bwt_vle_encode")
        return st

    def vle_encode(self, d_in, offsets, code, length, stream=None):
        """(stream uint8 trimmed to its bytes, byte_off int64[nb + 1], block_bits int64[nb]) CUDA tensors;
        code / length: uint32[256] / uint8[256] (numpy arrays or CUDA tensors)."""
        import torch
        dev = d_in.device
        d_code = code if isinstance(code, torch.Tensor) else torch.from_numpy(
            np.ascontiguousarray(code, dtype=np.uint32).view(np.int32)).to(dev)
        d_len = length if isinstance(length, torch.Tensor) else torch.from_numpy(
            np.ascontiguousarray(length, dtype=np.uint8)).to(dev)
        nb = (offsets.size if isinstance(offsets, np.ndarray) else offsets.numel()) - 1
        out = torch.empty(4 * d_in.numel() + 8, dtype=torch.uint8, device=dev)
        byte_off = torch.empty(nb + 1, dtype=torch.int64, device=dev)
        bits = torch.empty(nb, dtype=torch.int64, device=dev)
        self.vle_encode_into(d_in, offsets, d_code, d_len, out, byte_off, bits, stream)
        return out[:int(byte_off[nb].item())], byte_off, bits

    def mtf_encode_into(self, d_in, offsets, d_out, stream=None, raise_on_error=True) -> int:
        keep, off_ptr, nb = self._offsets(offsets)
        st = self.lib.bwt_mtf_encode(self.handle, _ptr(d_in), off_ptr, nb, _ptr(d_out), _stream_handle(stream))
        if raise_on_error:
            check(st, "bwt_mtf_encode")
        return st

    def mtf_encode(self, d_in, offsets, stream=None):
        import torch
        out = torch.empty_like(d_in)
        self.mtf_encode_into(d_in, offsets, out, stream)
        return out

    def stats(self) -> dict:
        s = Stats()
        check(self.lib.bwt_plan_stats(self.handle, ctypes.byref(s)), "bwt_plan_stats")
        return s.as_dict()

    def last_status(self) -> int:
        return self.lib.bwt_plan_last_status(self.handle)

    def set_radix(self, radix_bits: int, tile_keys: int) -> None:
        check(self.lib.bwt_plan_set_radix(self.handle, radix_bits, tile_keys), "bwt_plan_set_radix")

    def set_round_radix(self, radix_bits: int) -> None:
        check(self.lib.bwt_plan_set_round_radix(self.handle, radix_bits), "bwt_plan_set_round_radix")

    def autotune(self, d_in, offsets, d_L, d_primary, cache_path: str | None = None, repeats: int = 3,
                 stream=None) -> tuple[int, int, float]:
        """bwt_plan_autotune: returns (radix_bits, tile_keys, mean ms) and keeps them in the plan."""
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        rb, tk, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        check(self.lib.bwt_plan_autotune(self.handle, _ptr(d_in), off.ctypes.data, off.size - 1, _ptr(d_L),
                                         _ptr(d_primary), _stream_handle(stream),
                                         cache_path.encode() if cache_path else None, repeats, ctypes.byref(rb),
                                         ctypes.byref(tk), ctypes.byref(ms)), "bwt_plan_autotune")
        return rb.value, tk.value, ms.value

    def debug_waits(self, spin_limit: int, withhold_publish: bool) -> None:
        check(self.lib.bwt_plan_debug_waits(self.handle, spin_limit, int(withhold_publish)), "bwt_plan_debug_waits")


def bwt_inverse_check(L, primary: int, original) -> int:
    """Host check: BWT_OK if inverting L from `primary` reproduces `original`."""
    lib = _lib.load()
    L = np.ascontiguousarray(L, dtype=np.uint8)
    o = np.ascontiguousarray(original, dtype=np.uint8)
    if L.size != o.size:
        return _lib.BWT_EINVAL
    return lib.bwt_inverse_check(L.ctypes.data, L.size, int(primary), o.ctypes.data)
