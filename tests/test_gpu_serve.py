"""Serving loop with continuous batching: blocks of many streams of
different shapes, admitted by device memory (a budget small enough to force
queuing), batched into shared launches while others run.  Each block's result
must be the same alone and in the mix (bit for bit for complex int8), and a
stream's blocks must follow its own history (Section 4.1) in order."""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_08197_gb300 import lof, serve

pytestmark = pytest.mark.gpu


def _streams():
    shapes = [(1, 64, 1024), (2, 128, 2048), (1, 96, 4096), (3, 64, 1024), (2, 256, 1024),
              (1, 112, 8192)]
    return [serve.StreamSpec(i, S, C, T, period_s=0.05) for i, (S, C, T) in enumerate(shapes)]


def _results(srv):
    return {(r.spec.sid, r.block): (r.h_mask.numpy().copy(), r.h_out.numpy().copy())
            for r in srv.finished}


def test_mixed_equals_alone_and_memory_admission():
    streams = _streams()
    n_blocks = 3
    blocks = {}
    biggest = max(serve.Request(s, 0, 0.0, serve.make_block(s, 0)).device_bytes() for s in streams)
    budget = int(2.5 * biggest)  # at most two requests resident: forces queuing
    srv, wall = serve.run(streams, n_blocks, budget, accelerated=True, keep_results=True,
                          blocks=blocks)
    mixed = _results(srv)
    rep = serve.report(srv, wall)
    srv.close()
    assert rep["blocks"] == len(streams) * n_blocks
    assert rep["launches"] < rep["blocks"]  # some launches held several streams
    for s in streams:
        alone_srv, _ = serve.run([s], n_blocks, budget, accelerated=True, keep_results=True,
                                 blocks=blocks)
        alone = _results(alone_srv)
        alone_srv.close()
        for b in range(n_blocks):
            m1, o1 = mixed[(s.sid, b)]
            m2, o2 = alone[(s.sid, b)]
            assert np.array_equal(m1, m2), (s.sid, b, "mask")
            assert np.array_equal(o1, o2), (s.sid, b, "data")


def test_served_stream_follows_its_history_like_the_oracle():
    s = serve.StreamSpec(0, 1, 64, 1024, period_s=0.02)
    n_blocks = 10  # past history_min, so the history flagger is active
    blocks = {}
    srv, _ = serve.run([s], n_blocks, 1 << 26, accelerated=False, jitter_s=0.005,
                       keep_results=True, blocks=blocks)
    res = _results(srv)
    srv.close()
    p = oracle.default_params()
    hist = [oracle.History(s.C, p) for _ in range(s.n_units)]
    for b in range(n_blocks):
        x = blocks[(0, b)].numpy()
        for u in range(s.n_units):
            st, pol = divmod(u, 2)
            ref = oracle.flag_unit(p, x[st, pol], history=hist[u])
            hist[u].commit(0, ref["pending"], ref["has_pending"])
            assert np.array_equal(res[(0, b)][0][st, pol], ref["mask"]), (b, u)
            assert np.array_equal(res[(0, b)][1][st, pol], ref["out"]), (b, u)
