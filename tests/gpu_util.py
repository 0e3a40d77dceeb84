"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

FP64_RTOL = 1e-11     # FP64 path vs FP64 oracle (rounding order differs)
FP32_RTOL = 5e-6      # complex64 path vs FP64 oracle (single rounding ~6e-8 x log n growth)


def to_dev(torch, A, dtype):
    return torch.from_numpy(np.ascontiguousarray(A)).to(device="cuda", dtype=dtype)


def to_host(T):
    return T.detach().cpu().numpy().astype(np.complex128)


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))
