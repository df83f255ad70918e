"""Shared helpers of the GPU parity tests: host <-> device marshalling and the
comparison of packed outputs (including the untouched bytes past ceil(W/8))."""
import numpy as np

CANARY = 0xAB


def to_device(img: np.ndarray, W: int | None = None, misalign: int = 0):
    """Copy an (H, pitch) uint8 image to the GPU.  misalign > 0 shifts the
    base address by that many bytes (exercises the unaligned load path).
    Returns (tensor, W)."""
    import torch
    H, pitch = img.shape
    W = pitch if W is None else W
    if misalign:
        buf = torch.zeros((H, pitch + misalign), dtype=torch.uint8, device="cuda")
        buf[:, misalign:] = torch.from_numpy(np.ascontiguousarray(img)).cuda()
        t = buf[:, misalign:]
    else:
        t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    return t, W


def out_buffer(H: int, W: int, extra: int = 0):
    import torch
    return torch.full((H, (W + 7) // 8 + extra), CANARY, dtype=torch.uint8, device="cuda")


def check_packed(out, ref_packed: np.ndarray, W: int):
    """Bit-exact comparison of the first ceil(W/8) bytes of each row; bytes
    past them must keep the canary."""
    got = out.cpu().numpy()
    wb = (W + 7) // 8
    np.testing.assert_array_equal(got[:, :wb], ref_packed[:, :wb])
    if got.shape[1] > wb:
        assert (got[:, wb:] == CANARY).all(), "bytes past ceil(W/8) were written"


def unpack(packed: np.ndarray, W: int) -> np.ndarray:
    return np.unpackbits(packed, axis=1, bitorder="little")[:, :W]
