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


def xor_classes_dev(slots: torch.Tensor, alt_step: torch.Tensor) -> torch.Tensor:
    """Class codes (tag << 32 | min(j, alt)) of every nonzero slot of an
    (m, b) slot tensor under the XOR policy, sorted.  alt_step[t] = H(t) mod m
    for every tag value t, computed by the oracle (a torch gather and sort
    only; no value comes from the filter's kernels)."""
    s = slots.to(torch.int64)
    j, _ = torch.nonzero(s, as_tuple=True)
    t = s[s != 0]
    alt = j ^ alt_step[t]
    lo = torch.minimum(j, alt)
    return torch.sort((t << 32) | lo).values


def key_classes_dev(fp, i1, i2) -> torch.Tensor:
    """Sorted class codes (fp << 32 | min(i1, i2)) of keys, from the
    oracle's hashes (numpy arrays)."""
    lo = np.minimum(i1, i2).astype(np.int64)
    code = (fp.astype(np.int64) << 32) | lo
    return torch.sort(torch.from_numpy(code).cuda()).values


def alt_step_table(o, f: int) -> torch.Tensor:
    """H(t) mod m for every f-bit tag t (index 0 unused), from the oracle."""
    tab = np.zeros(1 << f, np.int64)
    for t in range(1, 1 << f):
        tab[t] = o.alt(0, t)
    return torch.from_numpy(tab).cuda()
