"""Failure detection without faulting the GPU: a kernel's bounded wait runs
out and reports a status, host-side waits time out cleanly, and the context
stays usable afterwards."""
import numpy as np
import pytest

import datagen as D
import oracle as O
from gpu_helpers import make_query, oracle_thresholds

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives():
    import torch

    import paper_2403_14902_b300 as H
    rc = H.load().hydro_selftest_bounded_wait(0, 2_000_000)    # 2 ms
    assert rc == H.ETIMEOUT
    assert b"as designed" in H.load().hydro_last_error()
    # the device still runs ordinary work
    w = D.workload("mlp3", n=256)
    th, _ = oracle_thresholds(w)
    q = make_query(w, th, batch=256)
    X = D.stream_tuples(w)
    words, counts, info = q.poll(q.submit(torch.from_numpy(X).cuda()))
    pm = O.pass_matrix(O.udf_scores("vec", X, D.predicate_weights(w)), th)
    assert np.array_equal(H.bits_from_words(words, 256), O.result_bits(pm))
    q.close()


def test_poll_without_wait_reports_eagain_or_result():
    import torch

    import paper_2403_14902_b300 as H
    w = D.workload("mlp3", n=256)
    th, _ = oracle_thresholds(w)
    q = make_query(w, th, batch=256)
    X = torch.from_numpy(D.stream_tuples(w)).cuda()
    bid = q.submit(X)
    try:
        q.poll(bid, wait_ms=0)          # may or may not be done yet
    except H.HydroError as e:
        assert e.status == H.EAGAIN
        q.poll(bid)                     # then a blocking poll returns it
    q.close()
