"""Continuous batching (npm_server_*): each request's result is the same
served alone and in a mix with others, admission respects the staging pool,
and training requests are ordered between queries."""
import threading

import numpy as np
import pytest

import synth
from gpu_helpers import cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _req(n, seed, rows=3):
    pos = torch.from_numpy(synth.positions(seed, n)).pin_memory()
    u = torch.from_numpy(synth.sample_uniforms(seed, n, rows=rows)).pin_memory()
    d = torch.empty((3, n)).pin_memory()
    p = torch.empty((n,)).pin_memory()
    return pos, u, d, p


@pytest.mark.parametrize("precision", [synth.FP32, synth.BF16X3])
def test_same_alone_and_in_the_mix(precision):
    import paper_2504_04315_gb300 as npm
    w = synth.TINY
    params = synth.random_params(w, 41)
    sizes = [5000, 777, 20000, 1, 4096, 12345]
    m = make_model(w, params, 1 << 16, precision=precision)
    # Reference: the direct device API, one request at a time.
    refs = []
    for i, n in enumerate(sizes):
        pos, u, _, _ = _req(n, 100 + i)
        d, p, _ = m.query_sample(pos.cuda(), u.cuda())
        refs.append((host(d), host(p)))
    with npm.Server(m, 1 << 16) as srv:
        alone = []
        for i, n in enumerate(sizes):
            r = _req(n, 100 + i)
            srv.wait(srv.submit_query(*r))
            alone.append((r[2].numpy().copy(), r[3].numpy().copy()))
        mixed = [_req(n, 100 + i) for i, n in enumerate(sizes)]
        # Queue them while admission is held, so that they share launches.
        srv.hold(True)
        tickets = [srv.submit_query(*r) for r in mixed]
        srv.hold(False)
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["max_requests_per_batch"] >= 2, st
    for i in range(len(sizes)):
        for a, b, c in zip(alone[i], (mixed[i][2].numpy(), mixed[i][3].numpy()), refs[i]):
            assert np.array_equal(a, b), i
            assert np.array_equal(a, c), i


def test_admission_by_memory_and_concurrent_submitters():
    import paper_2504_04315_gb300 as npm
    w = synth.TINY
    params = synth.random_params(w, 42)
    m = make_model(w, params, 1 << 14, precision=synth.FP32)
    pool = 8192
    reqs = [_req(6000 - 37 * i, 200 + i) for i in range(8)]
    refs = []
    for i, r in enumerate(reqs):
        d, p, _ = m.query_sample(r[0].cuda(), r[1].cuda())
        refs.append((host(d), host(p)))
    with npm.Server(m, pool) as srv:
        with pytest.raises(npm.NpmError) as e:
            big = _req(pool + 1, 9)
            srv.submit_query(*big)
        assert e.value.status == 4  # NPM_ERR_CAPACITY
        out = [None] * len(reqs)

        def client(k):
            for i in range(k, len(reqs), 2):
                out[i] = srv.wait(srv.submit_query(*reqs[i]))

        ths = [threading.Thread(target=client, args=(k,)) for k in range(2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        st = srv.stats()
    assert st["pool_peak_used"] <= pool
    assert st["requests_done"] == len(reqs)
    for i, r in enumerate(reqs):
        assert np.array_equal(r[2].numpy(), refs[i][0])
        assert np.array_equal(r[3].numpy(), refs[i][1])


def test_training_is_ordered_between_queries():
    import paper_2504_04315_gb300 as npm
    w = synth.TINY
    params = synth.random_params(w, 43)
    n = 4096
    m = make_model(w, params, n, precision=synth.FP32)
    q = _req(n, 300)
    d0, p0, _ = m.query_sample(q[0].cuda(), q[1].cuda())
    b = synth.train_batch_uniform(w, n, seed=301)
    tb = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (b.pos, b.dir, b.radiance, b.pdf)]
    q1 = _req(n, 300)
    q2 = _req(n, 300)
    with npm.Server(m, 3 * n) as srv:
        t1 = srv.submit_query(*q1)
        tt = srv.submit_train(*tb)
        t2 = srv.submit_query(*q2)
        for t in (t1, tt, t2):
            srv.wait(t)
        st = srv.stats()
    assert st["train_done"] == 1
    # Before the step: the original weights.
    assert np.array_equal(q1[2].numpy(), host(d0)) and np.array_equal(q1[3].numpy(), host(p0))
    # After the step: the trained weights, as the handle now holds them.
    d1, p1, _ = m.query_sample(q[0].cuda(), q[1].cuda())
    assert np.array_equal(q2[2].numpy(), host(d1)) and np.array_equal(q2[3].numpy(), host(p1))
    assert not np.array_equal(host(d1), host(d0))
