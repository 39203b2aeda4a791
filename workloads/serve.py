"""Device buffers for a serving trace (inputs only): each request's keys as
a device tensor slice and its flag buffer."""
from __future__ import annotations

from .gen import keys_dev


def materialize(sizes, plan, stream=None):
    """Generate the key streams of a `serve_trace` plan on the current CUDA
    device.  Returns (requests, keepalive) with requests[i] = (filter index,
    op, keys tensor, flags tensor)."""
    import torch

    sh = stream.cuda_stream if stream is not None else 0
    nf = len(sizes)
    ins_hi = [0] * nf
    neg_hi = [0] * nf
    for f, op, n, ps, pn, ns, nn in plan:
        ins_hi[f] = max(ins_hi[f], ps + pn)
        neg_hi[f] = max(neg_hi[f], ns + nn)
    keys_f, negs_f = [], []
    for f in range(nf):
        k = torch.empty(max(1, ins_hi[f]), dtype=torch.int64, device="cuda")
        if ins_hi[f]:
            keys_dev(k.data_ptr(), ins_hi[f], 10000 + f, 0, sh)
        g = torch.empty(max(1, neg_hi[f]), dtype=torch.int64, device="cuda")
        if neg_hi[f]:
            keys_dev(g.data_ptr(), neg_hi[f], 20000 + f, 0, sh)
        keys_f.append(k)
        negs_f.append(g)
    q_total = sum(n for _, op, n, *_ in plan if op == "contains")
    qbuf = torch.empty(max(1, q_total), dtype=torch.int64, device="cuda")
    flags = torch.zeros(max(1, sum(p[2] for p in plan)), dtype=torch.uint8, device="cuda")
    reqs = []
    qoff = foff = 0
    with torch.cuda.stream(stream) if stream is not None else _nullctx():
        for f, op, n, ps, pn, ns, nn in plan:
            if op == "contains":
                dst = qbuf[qoff:qoff + n]
                if pn:
                    dst[:pn].copy_(keys_f[f][ps:ps + pn])
                if nn:
                    dst[pn:].copy_(negs_f[f][ns:ns + nn])
                keys = dst
                qoff += n
            else:
                keys = keys_f[f][ps:ps + pn]
            reqs.append((f, op, keys, flags[foff:foff + n]))
            foff += n
    if stream is not None:
        stream.synchronize()
    else:
        torch.cuda.synchronize()
    return reqs, (keys_f, negs_f, qbuf, flags)


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
