"""GPU: the request server (continuous batching, admission by device memory).

* Batch invariance: every request's result is bit-identical to locc_detect of
  that request alone, while it shares launches with other requests (fp32,
  bf16 and fp8).  Each output row depends only on its own pair, so the stated
  tolerance for "alone vs in the mix" is zero.
* Admission: with an arena smaller than the sum of the requests, requests wait
  for memory and are admitted as blocks free up; the arena high-water mark
  stays within the budget; a request that can never fit is refused at submit;
  a full queue refuses with BUSY.
* Continuous batching: a small request submitted behind a large one finishes
  in one launch and before the large one.
* Host-side faults: bad indices are refused at submit; a client that never
  waits does not block shutdown.
"""

import threading
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 0.25
N_SHAPES = 16


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def lib():
    return synth.make_library(N_SHAPES, 3)


def _pinned(a):
    t = torch.empty(a.shape, dtype={np.float32: torch.float32, np.int32: torch.int32}[a.dtype.type],
                    pin_memory=True)
    out = t.numpy()
    out[...] = a
    return out


def _requests(sizes, seed):
    reqs = []
    for i, (n_env, n_pairs) in enumerate(sizes):
        p, s, q = synth.client_batch(N_SHAPES, n_env, n_pairs, seed + i, extent=0.6)
        reqs.append((_pinned(p), _pinned(s), _pinned(q)))
    return reqs


def _alone(det, req):
    dev = _dev()
    p, s, q = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in req)
    out = det.detect(p, s, q)
    det.status()
    return out.cpu().numpy()


def _out(n):
    return _pinned(np.zeros((n, 8), np.float32))


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_batch_invariance(lib, prec):
    from paper_2304_09439_b300 import Detector, Server
    _dev()
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(1, bias_scale=0.05), R, prec)
    sizes = [(64, 100), (300, 5000), (2000, 40000), (64, 1), (900, 12345), (128, 777),
             (5000, 60000), (100, 2500)]
    reqs = _requests(sizes, 100)
    want = [_alone(det, r) for r in reqs]
    with Server(det, max_batch_pairs=8192, max_active=64) as srv:
        outs = [_out(r[2].shape[0]) for r in reqs]
        ids = [None] * len(reqs)

        def client(k):
            for i in range(k, len(reqs), 3):
                ids[i] = srv.submit(*reqs[i], out=outs[i])

        th = [threading.Thread(target=client, args=(k,)) for k in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        infos = [srv.wait(i) for i in ids]
        st = srv.stats()
    for i, (w, o) in enumerate(zip(want, outs)):
        assert np.array_equal(w.view(np.uint32), o.view(np.uint32)), \
            f"request {i} ({sizes[i]}) differs alone vs in the mix"
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["pairs_completed"] == sum(n for _, n in sizes)
    # the mix really shared launches: some launch carried several requests
    assert sum(i["launches"] for i in infos) > st["launches"], (infos, st)
    assert max(i["launches"] for i in infos) >= 8  # 60000 pairs over 8192-pair launches
    det.close()


def test_admission_by_memory(lib):
    from paper_2304_09439_b300 import Detector, Server, LoccError
    _dev()
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(1), R, "bf16")
    sizes = [(200, 3000)] * 10
    reqs = _requests(sizes, 200)
    # inputs of one request: poses + shapes + pairs, each rounded to 256 B
    need = max(-(-r[0].nbytes // 256) * 256 + -(-r[1].nbytes // 256) * 256 +
               -(-r[2].nbytes // 256) * 256 for r in reqs)
    budget = 2 * need + need // 2  # two requests at a time
    want = [_alone(det, r) for r in reqs]
    with Server(det, arena_bytes=budget, max_batch_pairs=4096) as srv:
        outs = [_out(r[2].shape[0]) for r in reqs]
        ids = [srv.submit(*r, out=o) for r, o in zip(reqs, outs)]
        infos = [srv.wait(i) for i in ids]
        st = srv.stats()
        # larger than the whole arena: refused at once
        big = _requests([(4000, 200000)], 300)[0]
        with pytest.raises(LoccError) as e:
            srv.submit(*big, out=_out(big[2].shape[0]))
        assert e.value.code == -2
    for w, o in zip(want, outs):
        assert np.array_equal(w.view(np.uint32), o.view(np.uint32))
    assert st["arena_peak"] <= budget and st["arena_bytes"] <= budget
    assert st["max_active_seen"] == 2, st
    # later requests waited for memory: admission times grow along the queue
    assert infos[-1]["admit_us"] > infos[0]["admit_us"]
    det.close()


def test_queue_limit_busy(lib):
    from paper_2304_09439_b300 import Detector, Server, LoccError
    _dev()
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(1), R, "fp32")
    a, b = _requests([(2000, 100000), (100, 5000)], 400)
    need = sum(-(-x.nbytes // 256) * 256 for x in a)
    assert need >= sum(-(-x.nbytes // 256) * 256 for x in b)
    # `a` fills the arena for its whole run (~100k pairs on the fp32 path);
    # `b` queues behind it; a third request would exceed max_queued_pairs
    with Server(det, arena_bytes=need, max_batch_pairs=4096, max_queued_pairs=6000) as srv:
        oa, ob, oc = _out(100000), _out(5000), _out(5000)
        ia = srv.submit(*a, out=oa)
        time.sleep(0.005)
        ib = srv.submit(*b, out=ob)
        with pytest.raises(LoccError) as e:
            srv.submit(*b, out=oc)
        assert e.value.code == -7
        srv.wait(ia)
        srv.wait(ib)
        st = srv.stats()
    assert st["rejected"] == 1 and st["completed"] == 2
    assert np.array_equal(_alone(det, b).view(np.uint32), ob.view(np.uint32))
    det.close()


def test_small_request_overtakes_large(lib):
    from paper_2304_09439_b300 import Detector, Server
    _dev()
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(1), R, "fp32")
    big, small = _requests([(8000, 300000), (64, 200)], 500)
    with Server(det, max_batch_pairs=16384) as srv:
        ob, os_ = _out(300000), _out(200)
        t_big = time.perf_counter()
        ib = srv.submit(*big, out=ob)
        time.sleep(0.002)
        t_small = time.perf_counter()
        is_ = srv.submit(*small, out=os_)
        info_s = srv.wait(is_)
        info_b = srv.wait(ib)
    assert info_s["launches"] == 1
    assert info_b["launches"] >= 300000 // 16384
    assert t_small + info_s["done_us"] * 1e-6 < t_big + info_b["done_us"] * 1e-6
    assert np.array_equal(_alone(det, small).view(np.uint32), os_.view(np.uint32))
    det.close()


def test_bad_requests_and_shutdown(lib):
    from paper_2304_09439_b300 import Detector, Server, LoccError
    _dev()
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(1), R, "bf16")
    p, s, q = _requests([(50, 300)], 600)[0]
    srv = Server(det, max_batch_pairs=1024)
    bad = q.copy()
    bad[7, 1] = p.shape[0]
    with pytest.raises(LoccError) as e:
        srv.submit(p, s, bad)
    assert e.value.code == -1
    bs = s.copy()
    bs[3] = N_SHAPES
    with pytest.raises(LoccError) as e:
        srv.submit(p, bs, q)
    assert e.value.code == -1
    # empty request completes at once
    i0 = srv.submit(p, s, q[:0])
    assert srv.wait(i0, timeout_ms=1000)["launches"] == 0
    with pytest.raises(LoccError):
        srv.wait(123456789)
    # submitted, never waited for: shutdown finishes the work and returns
    o = _out(300)
    srv.submit(p, s, q, out=o)
    srv.close()
    assert np.array_equal(_alone(det, (p, s, q)).view(np.uint32), o.view(np.uint32))
    det.close()


def test_launch_pressure_bounds_admission(lib):
    # many large requests: each counts up to one launch (max_batch_pairs) of
    # pressure, so only a few are admitted at once (more only as the admitted
    # ones near their end); a small request is still admitted beside them
    from paper_2304_09439_b300 import Detector, Server
    _dev()
    det = Detector(lib.points, lib.aabb, synth.xavier_weights(1), R, "bf16")
    big = _requests([(2000, 40000)] * 12, 700)
    small = _requests([(64, 150)], 800)[0]
    with Server(det, max_batch_pairs=8192, max_active_pairs=4 * 8192) as srv:
        outs = [_out(40000) for _ in big]
        ids = [srv.submit(*r, out=o) for r, o in zip(big, outs)]
        o_s = _out(150)
        i_s = srv.submit(*small, out=o_s)
        infos = [srv.wait(i) for i in ids]
        info_s = srv.wait(i_s)
        st = srv.stats()
    assert 2 <= st["max_active_seen"] <= 8, st  # without the bound all 13 would be
    assert info_s["launches"] == 1
    for r, o in zip(big[:2], outs[:2]):
        assert np.array_equal(_alone(det, r).view(np.uint32), o.view(np.uint32))
    det.close()
