"""lof_flag_block_noalloc: the allocation-free entry point for callers that
may not allocate memory while they run (real-time threads, fixed memory
budgets).  Its results must equal those of lof_flag_block -- bit for bit for
integer voltages -- on consecutive calls that share its static scratch, for
every input type and option it accepts; blocks that do not fit its fixed
scratch, and capturing streams, are refused before anything is enqueued."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, synth

from helpers import compare_unit

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


def _stokes(seed, C, T):
    spec = synth.PulsarSpec(n_subband=1, C=C, T=T)
    return synth.stokes_block(spec, seed=seed, block=0, device="cpu")[0].numpy().astype(np.float32)


def _run(datas, entry, fl=None, params=None):
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
        rc = lof.lof_flag_block_noalloc(params or lof.lof_default_params(), dt, units, st.data_ptr(),
                                        stream.cuda_stream)
        assert rc == lof.LOF_OK, lof.lof_last_error()
        stream.synchronize()
        status = int(st.item())
    return [o.cpu().numpy() for o in outs], [m.cpu().numpy() for m in masks], stats.cpu(), status


def _same(a, b):
    """Bit-identical arrays (float data compared by their bits)."""
    if a.dtype == np.float32:
        return np.array_equal(a.view(np.uint32), b.view(np.uint32))
    return np.array_equal(a, b)


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


def test_noalloc_float32_units_match_lof_flag_block_and_oracle_statistics():
    """Stokes I units (the float kernel, no unit-state scratch) on two calls."""
    with lof.Flagger(0) as fl:
        for call, seed in enumerate((31, 32)):
            datas = [_stokes(seed, 16, 12288), _stokes(seed + 100, 13, 1000)]
            o_ref, m_ref, s_ref, _ = _run(datas, "ctx", fl)
            o, m, s, status = _run(datas, "noalloc")
            assert status == 0
            for i, d in enumerate(datas):
                assert _same(m[i], m_ref[i]) and _same(o[i], o_ref[i]), f"call {call} unit {i}"
                g = lof.decode_stats(s[i])
                assert g == lof.decode_stats(s_ref[i])
                want = oracle.flag_unit(oracle.default_params(), d)["stats"]
                for k in ("median_f", "sigma_f", "median_t", "sigma_t"):
                    assert abs(g[k] - want[k]) <= 1e-6 * max(abs(want[k]), 1e-30), (k, g[k], want[k])


def test_noalloc_exact_statistics_option_with_sir_matches_oracle():
    """The integrated time mode (exact-statistics unit kernel) plus the SIR
    pass: bit-exact against the oracle and lof_flag_block, two calls."""
    kw = dict(time_mode=lof.LOF_TIME_INTEGRATED, sir_percent=20)
    P = oracle.default_params(time_mode=1, sir_percent=20)
    with lof.Flagger(0, **kw) as fl:
        for call, seed in enumerate((303, 404)):
            datas = _block(seed, lof.LOF_CI16)
            o_ref, m_ref, s_ref, _ = _run(datas, "ctx", fl)
            o, m, s, status = _run(datas, "noalloc", params=lof.lof_default_params(**kw))
            assert status == 0
            for i, d in enumerate(datas):
                assert np.array_equal(m[i], m_ref[i]) and np.array_equal(o[i], o_ref[i])
                compare_unit(d, oracle.flag_unit(P, d), torch.as_tensor(o[i]), torch.as_tensor(m[i]),
                             s[i], tag=f"call {call} unit {i}")


def test_noalloc_rejects_history_oversized_blocks_and_capture():
    x = torch.zeros((4, 64, 2), dtype=torch.int16, device=DEV)
    u = lof.make_unit(x, None, None, history_slot=0)
    stream = torch.cuda.current_stream().cuda_stream
    assert lof.lof_flag_block_noalloc(None, lof.LOF_CI16, [u], 0, stream) == lof.LOF_ERR_INVALID
    assert "history" in lof.lof_last_error()
    many = [lof.make_unit(x) for _ in range(1025)]
    assert lof.lof_flag_block_noalloc(None, lof.LOF_CI16, many, 0, stream) == lof.LOF_ERR_INVALID
    assert "maximum" in lof.lof_last_error()
    # long rows need more general-path scratch than the static array holds
    y = torch.zeros((1, 200000, 2), dtype=torch.int16, device=DEV)
    long_rows = [lof.make_unit(y) for _ in range(100)]
    assert lof.lof_flag_block_noalloc(None, lof.LOF_CI16, long_rows, 0, stream) == lof.LOF_ERR_INVALID
    assert "scratch" in lof.lof_last_error()
    # a capturing stream: refused, nothing enqueued (the capture stays empty)
    ok = [lof.make_unit(x)]
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = lof.lof_flag_block_noalloc(None, lof.LOF_CI16, ok, 0, side.cuda_stream)
    assert rc == lof.LOF_ERR_INVALID and "capturing" in lof.lof_last_error()
    torch.cuda.synchronize()
    # and the entry point still works afterwards
    st = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    assert lof.lof_flag_block_noalloc(None, lof.LOF_CI16, ok, st.data_ptr(), stream) == lof.LOF_OK
    torch.cuda.synchronize()
    assert int(st.item()) == 0
