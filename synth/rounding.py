"""Rounding of inputs to the storage precisions of the mixed paths.

The mixed-precision solver stores matrix values in FP32 and (optionally) the POD
basis in BF16; the system it solves is the one with those rounded entries. Tests
hand both the oracle and the CUDA path the rounded arrays (as float64), so that
both solve the same system.
"""
import numpy as np


def round_f32(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(a) -> np.ndarray:
    """Round float64 values to the nearest BF16 (ties to even on the float64 significand)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    u = a.view(np.uint64)
    keep = ~np.uint64(0x00001FFFFFFFFFFF)
    r = (u + np.uint64(0x00001FFFFFFFFFFF) + ((u >> np.uint64(45)) & np.uint64(1))) & keep
    out = r.view(np.float64).astype(np.float32).astype(np.float64)
    return np.where(np.isfinite(a), out, a)


def round_phi(phi, phi_dtype: str) -> np.ndarray:
    if phi_dtype == "f64":
        return np.asarray(phi, dtype=np.float64)
    if phi_dtype == "f32":
        return round_f32(phi)
    if phi_dtype == "bf16":
        return round_bf16(phi)
    raise ValueError(phi_dtype)
