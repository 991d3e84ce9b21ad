"""Shared test helpers: run a block through the CUDA library and the oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_1701_08197_gb300 import lof

PARAM_NAMES = ["p", "sensitivity", "start_threshold", "max_window", "history_len", "history_min",
               "history_k", "sigma_estimator", "enable_freq", "enable_time", "enable_history"]


def oracle_params(**kw):
    return oracle.default_params(**kw)


def gpu_units(datas, dev, with_out=True, with_mask=True, slots=None, inplace=False):
    """Device copies + output buffers + descriptors for a list of host arrays."""
    ins, outs, masks, units = [], [], [], []
    stats = lof.stats_tensor(len(datas), dev)
    off = 0
    for i, d in enumerate(datas):
        x = torch.as_tensor(d).to(dev)
        C, T = d.shape[0], d.shape[1]
        o = x if inplace else (torch.full_like(x, 77) if with_out else None)
        m = torch.full((C, T), 9, dtype=torch.uint8, device=dev) if with_mask else None
        slot = -1 if slots is None else slots[i]
        units.append(lof.make_unit(x, o, m, slot, stats[i]))
        ins.append(x)
        outs.append(o)
        masks.append(m)
        off += C
    return ins, outs, masks, stats, units


def compare_unit(d, r_oracle, out_gpu, mask_gpu, stats_gpu, tag=""):
    """Bit-exact comparison of one integer unit."""
    m = mask_gpu.cpu().numpy()
    assert np.array_equal(m, r_oracle["mask"]), (
        f"{tag}: mask mismatch at {np.argwhere(m != r_oracle['mask'])[:10].tolist()} "
        f"(gpu ones {int(m.sum())}, oracle ones {int(r_oracle['mask'].sum())})")
    if out_gpu is not None:
        o = out_gpu.cpu().numpy()
        assert np.array_equal(o, r_oracle["out"]), f"{tag}: output data mismatch"
    if stats_gpu is not None:
        g = lof.decode_stats(stats_gpu)
        s = r_oracle["stats"]
        for k in s:
            assert g[k] == s[k], f"{tag}: stats {k}: gpu {g[k]!r} oracle {s[k]!r}"
