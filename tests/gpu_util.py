"""Helpers for the GPU tests: numpy <-> CUDA tensors and bank repacking."""
import numpy as np
import torch

_VIEW = {np.dtype(np.uint32): np.int32, np.dtype(np.uint16): np.int16}


def dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype in _VIEW:
        a = a.view(_VIEW[a.dtype])
    return torch.from_numpy(a).cuda()


def host(t: torch.Tensor, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def pack_rows(bank_bytes: np.ndarray, row_words: int) -> np.ndarray:
    """Oracle byte-per-bit bank (n_bins, 4^q) -> bin-major u32 rows, bit t
    in bit t&31 of word t>>5, rows zero-padded to row_words."""
    nb, nbits = bank_bytes.shape
    out = np.zeros((nb, row_words * 32), dtype=np.uint8)
    out[:, :nbits] = bank_bytes
    packed = np.packbits(out, axis=1, bitorder="little")  # byte k holds bits 8k..8k+7
    return packed.view("<u4").reshape(nb, row_words)
