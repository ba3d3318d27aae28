"""Shared test helpers (comparison metrics only; no method arithmetic)."""
import numpy as np


def ordered_f32(a):
    """Map float32 bit patterns to integers whose order and spacing follow the
    floats (adjacent floats differ by 1; +0 and -0 both map to 0)."""
    i = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    return np.where(i < 0, -(i & 0x7FFFFFFF), i)


def ulp_distance_f32(gpu, ref64):
    """Ordered-integer distance between FP32 results and FP64 references
    rounded to FP32 (round to nearest)."""
    return np.abs(ordered_f32(gpu) - ordered_f32(np.asarray(ref64, np.float64).astype(np.float32)))


def to_numpy(t):
    """Copy a CUDA tensor to host numpy; int32 storage of u32 words is viewed as uint32."""
    import torch

    a = t.detach().cpu().numpy()
    if t.dtype == torch.int32:
        a = a.view(np.uint32)
    return a
