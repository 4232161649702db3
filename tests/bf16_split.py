"""Round-to-nearest-even FP32 -> bf16 on the integer bits, and the hi/lo split of
the tensor-core pass's features (hi = RN(F), lo = RN(F - hi)), for the tests."""
import numpy as np


def rn_bf16_bits(f: np.ndarray) -> np.ndarray:
    """bf16 bit patterns (uint16) of FP32 values, round to nearest, ties to even
    (finite inputs)."""
    b = np.ascontiguousarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    return ((b + 0x7FFF + lsb) >> 16).astype(np.uint16)


def bf16_value(h: np.ndarray) -> np.ndarray:
    return (h.astype(np.uint32) << 16).view(np.float32)


def split_pair(F: np.ndarray):
    """(hi, lo) bit patterns with hi = RN(F) and lo = RN(F - hi); F - hi is exact in FP32."""
    F = np.asarray(F, dtype=np.float32)
    hi = rn_bf16_bits(F)
    lo = rn_bf16_bits((F - bf16_value(hi)).astype(np.float32))
    return hi, lo
