"""lof_flag_block_noalloc: the allocation-free entry point for callers that
may not allocate memory while they run (real-time threads, fixed memory
budgets).  Its results must equal those of lof_flag_block -- bit for bit for
integer voltages -- on consecutive calls that share its static scratch."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1701_08197_gb300 import lof, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _block(seed, dtype):
    rng = np.random.default_rng(seed)
    npdt = np.int8 if dtype == lof.LOF_CI8 else np.int16
    sigma = 8.0 if dtype == lof.LOF_CI8 else 32.0
    datas = []
    for C, T in [(256, 768), (64, 3072), (17, 1000), (5, 33)]:
        x = np.round(rng.normal(0, sigma, (C, T, 2)))
        x[rng.integers(0, C), :, 0] += 20 * sigma
        t0 = rng.integers(0, max(1, T - 20))
        x[:, t0:t0 + 10, 1] += 30 * sigma
        info = np.iinfo(npdt)
        datas.append(np.clip(x, info.min, info.max).astype(npdt))
    return datas


def _run(datas, entry, fl=None):
    ins = [torch.as_tensor(d).to(DEV) for d in datas]
    outs = [torch.full_like(x, 99) for x in ins]
    masks = [torch.full(x.shape[:2], 7, dtype=torch.uint8, device=DEV) for x in ins]
    stats = lof.stats_tensor(len(datas), DEV)
    units = [lof.make_unit(x, o, m, -1, stats[i]) for i, (x, o, m) in enumerate(zip(ins, outs, masks))]
    dt = lof.dtype_of(ins[0])
    stream = torch.cuda.current_stream()
    if entry == "ctx":
        fl.flag_block(dt, units, 0, stream)
        fl.status(stream)
        status = 0
    else:
        st = torch.full((1,), -1, dtype=torch.int32, device=DEV)
        rc = lof.lof_flag_block_noalloc(lof.lof_default_params(), dt, units, st.data_ptr(),
                                        stream.cuda_stream)
        assert rc == lof.LOF_OK, lof.lof_last_error()
        stream.synchronize()
        status = int(st.item())
    return [o.cpu().numpy() for o in outs], [m.cpu().numpy() for m in masks], stats.cpu(), status


@pytest.mark.parametrize("dtype", [lof.LOF_CI16, lof.LOF_CI8])
def test_noalloc_matches_lof_flag_block_on_two_calls(dtype):
    with lof.Flagger(0) as fl:
        for call, seed in enumerate((101, 202)):  # two calls in a row, different data
            datas = _block(seed, dtype)
            o_ref, m_ref, s_ref, _ = _run(datas, "ctx", fl)
            o, m, s, status = _run(datas, "noalloc")
            assert status == 0, f"call {call}: device status {status}"
            for i in range(len(datas)):
                assert np.array_equal(m[i], m_ref[i]), f"call {call} unit {i}: mask differs"
                assert np.array_equal(o[i], o_ref[i]), f"call {call} unit {i}: data differs"
                assert lof.decode_stats(s[i]) == lof.decode_stats(s_ref[i]), f"call {call} unit {i}"
            assert sum(int(x.sum()) for x in m) > 0


def test_noalloc_rejects_history_and_oversized_blocks():
    x = torch.zeros((4, 64, 2), dtype=torch.int16, device=DEV)
    u = lof.make_unit(x, None, None, history_slot=0)
    stream = torch.cuda.current_stream().cuda_stream
    assert lof.lof_flag_block_noalloc(None, lof.LOF_CI16, [u], 0, stream) == lof.LOF_ERR_INVALID
    assert "history" in lof.lof_last_error()
    many = [lof.make_unit(x) for _ in range(1025)]
    assert lof.lof_flag_block_noalloc(None, lof.LOF_CI16, many, 0, stream) == lof.LOF_ERR_INVALID
    assert "maximum" in lof.lof_last_error()
