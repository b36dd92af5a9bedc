"""Shared helpers of the GPU parity tests (inputs to the device, results back,
comparison against the oracle)."""

import numpy as np
import torch


def dev(a) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.int32))).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def inst_dev(inst, share_self: bool = True):
    """Device columns of an instance; a self-join's S columns are R's tensors
    (the library then maps once) unless share_self is False."""
    rk, rv = dev(inst.r_key), dev(inst.r_val)
    if inst.self_join and share_self:
        return rk, rv, rk, rv
    return rk, rv, dev(inst.s_key), dev(inst.s_val)


def rows_of(out_x: torch.Tensor, out_z: torch.Tensor, xs: np.ndarray, out_c: torch.Tensor | None = None):
    """The (x, z[, c]) rows of a sorted device result whose x is in xs, as host
    arrays (x values need not be present)."""
    xs = np.sort(np.unique(np.asarray(xs, np.int32)))
    q = torch.from_numpy(xs).to(out_x.device)
    lo = torch.searchsorted(out_x, q, right=False)
    hi = torch.searchsorted(out_x, q, right=True)
    lo, hi = host(lo), host(hi)
    parts_x, parts_z, parts_c = [], [], []
    for a, b in zip(lo, hi):
        if b > a:
            parts_x.append(host(out_x[a:b]))
            parts_z.append(host(out_z[a:b]))
            if out_c is not None:
                parts_c.append(host(out_c[a:b]))
    cat = (lambda p: np.concatenate(p) if p else np.zeros(0, np.int32))
    return cat(parts_x), cat(parts_z), (cat(parts_c) if out_c is not None else None)


def check_sorted_distinct(out_x: torch.Tensor, out_z: torch.Tensor, chunk: int = 1 << 28):
    """Strictly increasing (x, z) pairs, checked on the device in chunks."""
    n = out_x.numel()
    for a in range(0, max(n - 1, 0), chunk):
        b = min(n - 1, a + chunk)
        x0, x1 = out_x[a:b], out_x[a + 1:b + 1]
        z0, z1 = out_z[a:b], out_z[a + 1:b + 1]
        ok = (x1 > x0) | ((x1 == x0) & (z1 > z0))
        assert bool(ok.all()), f"order broken in [{a}, {b})"
