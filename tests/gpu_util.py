"""Host <-> device helpers for the GPU tests (64-bit words kept as int64)."""
import numpy as np
import torch


def dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def empty(*shape) -> torch.Tensor:
    return torch.empty(shape, dtype=torch.int64, device="cuda")
