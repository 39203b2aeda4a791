"""Helpers shared by the GPU tests (host <-> device key arrays)."""
import numpy as np
import torch


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def to_host_u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def to_host_u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def oracle_policy(policy: str) -> int:
    return {"xor": 0, "offset": 1}[policy]


def m_for(policy: str, m_xor: int) -> int:
    """A bucket count valid for the policy: the power of two for XOR, a
    nearby odd number for Offset (which allows any m)."""
    return m_xor if policy == "xor" else m_xor - 37
