"""Helpers shared by the GPU parity tests (host <-> device marshalling only)."""
import numpy as np
import torch

# numpy key dtype -> (torch container dtype, key_type for the C ABI)
KEYS = {
    np.dtype(np.int32): (torch.int32, "i32"),
    np.dtype(np.uint32): (torch.int32, "u32"),
    np.dtype(np.int64): (torch.int64, "i64"),
    np.dtype(np.uint64): (torch.int64, "u64"),
}
SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64,
          np.dtype(np.int32): np.int32, np.dtype(np.int64): np.int64,
          np.dtype(np.float32): np.float32, np.dtype(np.float64): np.float64}


def dev(a: np.ndarray, device="cuda") -> torch.Tensor:
    """Copy a numpy array to the device keeping its bits (unsigned -> signed container)."""
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(SIGNED[a.dtype])).to(device)


def host(t: torch.Tensor, dtype) -> np.ndarray:
    """Device tensor -> numpy array reinterpreted as `dtype` (same width)."""
    return t.detach().cpu().numpy().view(dtype)


def key_type(a: np.ndarray) -> str:
    return KEYS[np.dtype(a.dtype)][1]


def sorted_keys(rng, size, dtype, spread=None):
    info = np.iinfo(dtype)
    if spread is None:
        x = rng.integers(info.min, info.max, size=size, dtype=dtype, endpoint=True)
    else:
        base = rng.integers(info.min, info.max - spread, dtype=dtype, endpoint=True)
        x = rng.integers(0, spread, size=size, dtype=dtype) + base
    return np.sort(x, kind="stable")


def same_bits(a: np.ndarray, b: np.ndarray) -> bool:
    return a.shape == b.shape and a.tobytes() == b.tobytes()


def save_shapes(lib, code, vb):
    """Tile shape of every class (balanced, skewed, small, batched, pass) of
    a key type and payload width, for restore_shapes."""
    return [lib.cr_get_tile_shape_for(code, vb, c) for c in range(5)]


def restore_shapes(lib, code, vb, saved):
    for c, s in enumerate(saved):
        assert lib.cr_set_tile_shape_for(code, vb, c, s) == 0
