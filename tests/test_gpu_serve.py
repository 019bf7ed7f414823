"""Serving: persistent-kernel continuous batching through the C ABI.

Results equal the FP64 oracle (same tolerances as the batched kernels); each
request's result is bit-identical alone and inside a mix of concurrent
requests of other robots and ops; admission follows the HBM budget; the
kernel's bounded idle wait ends it and the next request relaunches it; host
waits time out with FRAX_ETIMEOUT instead of hanging."""

import time

import numpy as np
import pytest

import gen
import paper_2604_04310_gb300 as fx
from oracle import derivatives as dv
from oracle import rbd
from paper_2604_04310_gb300.serving import Server
from tests.pins import normwise

pytestmark = pytest.mark.gpu

ROBOTS = [gen.chain7(0), gen.humanoid(0), gen.random_tree(105), gen.random_tree(7, 64)]


def _inputs(robot, op, B, seed):
    s = gen.draw_states(robot, B, seed).as_f32()
    g = gen.draw_gbar(robot.nv, B, seed + 1).astype(np.float32).astype(np.float64)
    arrays = {"rnea": [s.q, s.qd, s.qdd], "crba": [s.q], "aba": [s.q, s.qd, s.tau],
              "rnea_grad": [s.q, s.qd, s.qdd, g]}[op]
    return s, g, [gen.to_soa(a) for a in arrays]


def _oracle(robot, op, s, g):
    if op == "rnea":
        return [rbd.rnea(robot, s.q, s.qd, s.qdd)]
    if op == "crba":
        return [rbd.crba(robot, s.q).reshape(s.B, -1)]
    if op == "aba":
        return [rbd.aba(robot, s.q, s.qd, s.tau)]
    return list(dv.rnea_vjp(robot, s.q, s.qd, s.qdd, g))


def _tol(robot, op):
    return 1e-3 if (op in ("aba", "rnea_grad") and robot.name != "chain7") or op == "rnea_grad" else 1e-4


@pytest.fixture(scope="module")
def server():
    srv = Server(budget_bytes=512 << 20, idle_exit_ms=20.0)
    models = [fx.Model.from_robot(r) for r in ROBOTS]
    ids = [srv.add_model(m) for m in models]
    yield srv, ids
    srv.close(force=True)


def _run(srv, mid, op, inputs, B, timeout_s=20.0):
    req = srv.submit(mid, op, inputs, B)
    assert req is not None
    t_end = time.time() + timeout_s
    while not srv.poll(req):
        assert time.time() < t_end, "request did not complete"
        time.sleep(1e-4)
    return srv.collect(req, mid, op, B)


@pytest.mark.parametrize("k", range(len(ROBOTS)))
@pytest.mark.parametrize("op", ["rnea", "crba", "aba", "rnea_grad"])
def test_served_results_match_oracle(server, k, op):
    srv, ids = server
    robot = ROBOTS[k]
    B = 200 if robot.n_bodies < 64 else 64
    s, g, inputs = _inputs(robot, op, B, 300 + k)
    outs, lat = _run(srv, ids[k], op, inputs, B)
    assert lat > 0
    for o, ref in zip(outs, _oracle(robot, op, s, g)):
        assert normwise(gen.from_soa(o, B), ref) < _tol(robot, op)


def test_alone_equals_in_the_mix(server):
    """A request computed alone and inside a stream of 60 concurrent requests
    (all robots, all ops, 1-4096 instances) gives bit-identical results."""
    srv, ids = server
    robot, mid = ROBOTS[1], ids[1]
    B = 777
    _, _, probe_in = _inputs(robot, "aba", B, 901)
    alone, _ = _run(srv, mid, "aba", probe_in, B)
    _, _, probe_g = _inputs(robot, "rnea_grad", 300, 902)
    alone_g, _ = _run(srv, mid, "rnea_grad", probe_g, 300)
    rng = np.random.default_rng(3)
    pending = {}  # request -> (model id, op, B)
    results = {}

    def drain_one():
        r = srv.wait_any(10000.0)
        assert r is not None
        m, op, Bp = pending.pop(r)
        results[r], _ = srv.collect(r, m, op, Bp)

    def submit(m, op, inp, Bp):
        req = srv.submit(m, op, inp, Bp)
        while req is None:  # budget or ring full: finish one and retry
            drain_one()
            req = srv.submit(m, op, inp, Bp)
        pending[req] = (m, op, Bp)
        return req

    probes = {}
    for j in range(60):
        if j == 25:
            probes["aba"] = submit(mid, "aba", probe_in, B)
        if j == 40:
            probes["rnea_grad"] = submit(mid, "rnea_grad", probe_g, 300)
        k = int(rng.integers(len(ROBOTS)))
        op = ["rnea", "crba", "aba", "rnea_grad"][int(rng.integers(4))]
        Bj = int(np.clip(np.exp(rng.uniform(0, np.log(4096))), 1, 4096))
        if ROBOTS[k].n_bodies == 64:
            Bj = min(Bj, 512)
        _, _, inp = _inputs(ROBOTS[k], op, Bj, 1000 + j)
        submit(ids[k], op, inp, Bj)
    while pending:
        drain_one()
    assert np.array_equal(results[probes["aba"]][0], alone[0])
    for a, b in zip(results[probes["rnea_grad"]], alone_g):
        assert np.array_equal(a, b)
    assert srv.info()["in_flight"] == 0


def test_admission_by_budget():
    robot = ROBOTS[0]
    srv = Server(budget_bytes=1 << 20, idle_exit_ms=20.0)
    mid = srv.add_model(fx.Model.from_robot(robot))
    # 7 + 7 + 7 + 7 rows x 4 B x B > 1 MiB for B = 16384: never admissible
    _, _, big = _inputs(robot, "rnea", 16384, 5)
    with pytest.raises(fx.FraxError) as e:
        srv.submit(mid, "rnea", big, 16384)
    assert e.value.status == 3  # FRAX_ENOMEM
    # fill the budget with admissible requests until the server says busy
    _, _, small = _inputs(robot, "crba", 1024, 6)  # 7 + 49 rows x 4 KiB = 224 KiB
    reqs = []
    while True:
        r = srv.submit(mid, "crba", small, 1024)
        if r is None:
            break
        reqs.append(r)
        assert len(reqs) < 10
    assert len(reqs) == 4 and srv.info()["bytes_in_use"] <= 1 << 20
    for r in reqs:
        while not srv.poll(r):
            time.sleep(1e-4)
        srv.collect(r, mid, "crba", 1024)
    assert srv.info()["bytes_in_use"] == 0
    assert srv.submit(mid, "crba", small, 1024) is not None  # admitted again
    srv.close(force=True)


def test_idle_exit_relaunch_and_timeouts():
    robot = ROBOTS[1]
    srv = Server(budget_bytes=1 << 30, idle_exit_ms=5.0)
    mid = srv.add_model(fx.Model.from_robot(robot))
    s, g, inp = _inputs(robot, "rnea", 64, 7)
    outs, _ = _run(srv, mid, "rnea", inp, 64)
    time.sleep(0.1)  # the kernel's bounded idle wait runs out; it exits
    l0 = srv.info()["kernel_launches"]
    outs2, _ = _run(srv, mid, "rnea", inp, 64)
    assert srv.info()["kernel_launches"] == l0 + 1
    assert np.array_equal(outs[0], outs2[0])
    assert normwise(gen.from_soa(outs2[0], 64), rbd.rnea(robot, s.q, s.qd, s.qdd)) < 1e-4
    # a host wait with nothing completing in time reports FRAX_ETIMEOUT
    B = 1 << 20  # ~3 ms of work: still in flight when the next two calls run
    _, _, big = _inputs(robot, "aba", B, 8)
    req = srv.submit(mid, "aba", big, B)
    assert srv.wait_any(0.0) is None
    # destroying with work in flight is refused unless forced
    with pytest.raises(fx.FraxError) as e:
        srv.close(force=False)
    assert e.value.status == 5  # FRAX_EBUSY
    while not srv.poll(req):
        time.sleep(1e-4)
    srv.collect(req, mid, "aba", B)
    assert srv.info()["device_status"] == 0
    srv.close()


def test_ring_full_and_bad_arguments():
    robot = ROBOTS[0]
    srv = Server(budget_bytes=64 << 20, idle_exit_ms=20.0)
    mid = srv.add_model(fx.Model.from_robot(robot))
    _, _, inp = _inputs(robot, "rnea", 1, 9)
    reqs = []
    for _ in range(1024):
        r = srv.submit(mid, "rnea", inp, 1)
        assert r is not None
        reqs.append(r)
    assert srv.submit(mid, "rnea", inp, 1) is None  # all ring slots hold uncollected requests
    with pytest.raises(fx.FraxError):
        srv.submit(mid + 5, "rnea", inp, 1)
    for r in reqs:
        while not srv.poll(r):
            time.sleep(1e-5)
        srv.collect(r, mid, "rnea", 1)
    assert srv.info()["completed"] == 1024
    srv.close()


def test_budget_larger_than_device_is_refused():
    with pytest.raises(fx.FraxError) as e:
        Server(budget_bytes=1 << 50)
    assert e.value.status == 3


def test_native_replay(server):
    """frax_server_replay: a Poisson-timed trace of mixed requests comes back
    with every latency measured and the same results as served one by one."""
    srv, ids = server
    rng = np.random.default_rng(11)
    trace, refs = [], []
    for j in range(40):
        k = int(rng.integers(len(ROBOTS)))
        op = ["rnea", "crba", "aba", "rnea_grad"][int(rng.integers(4))]
        Bj = int(np.clip(np.exp(rng.uniform(0, np.log(1024))), 1, 1024))
        _, _, inp = _inputs(ROBOTS[k], op, Bj, 5000 + j)
        trace.append((ids[k], op, inp))
        refs.append((ids[k], op, inp, Bj))
    arrival = np.cumsum(rng.exponential(200.0, size=len(trace)))
    lat, outs = srv.replay(trace, arrival, keep_outputs=True)
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    for (mid, op, inp, Bj), o in zip(refs[:12], outs[:12]):
        alone, _ = _run(srv, mid, op, inp, Bj)
        for a, b in zip(o, alone):
            assert np.array_equal(a, b)
    assert srv.info()["in_flight"] == 0


def test_long_mixed_replay_with_relaunches():
    """20 000 mixed requests (four robots, four ops, 1-4096 instances
    log-uniform) in four bursts separated by pauses longer than the idle
    limit, so the persistent kernel both runs for long stretches and exits
    and is relaunched between bursts. Every request completes, no device
    error is recorded, and sampled results match the FP64 oracle."""
    srv = Server(budget_bytes=1 << 30, idle_exit_ms=100.0)
    ids = [srv.add_model(fx.Model.from_robot(r)) for r in ROBOTS]
    rng = np.random.default_rng(77)
    pool = {}  # a few input sets per (robot, op, size class), reused across the trace
    trace, meta = [], []
    n, bursts = 20000, 4
    sizes = np.array([1, 2, 5, 13, 33, 90, 250, 700, 1900, 4096])
    for j in range(n):
        k = int(rng.integers(len(ROBOTS)))
        op = ["rnea", "crba", "aba", "rnea_grad"][int(rng.integers(4))]
        # log-uniform size, snapped to one of ten classes so a small pool of
        # input sets serves the whole trace
        Bj = int(sizes[np.abs(np.log(sizes) - rng.uniform(0, np.log(4096))).argmin()])
        if ROBOTS[k].n_bodies >= 64:
            Bj = min(Bj, 512)
        key = (k, op, Bj, j % 2)
        if key not in pool:
            pool[key] = _inputs(ROBOTS[k], op, Bj, 9000 + len(pool))
        trace.append((ids[k], op, pool[key][2]))
        meta.append(key)
    per = n // bursts
    gaps = rng.exponential(1e6 / 20000.0, size=n)  # about 20 000 requests/s inside a burst
    for b in range(1, bursts):
        gaps[b * per] += 250e3  # 250 ms pauses: longer than idle_exit_ms
    arrival = np.cumsum(gaps)
    keep = set(int(x) for x in rng.choice(n, 24, replace=False))
    lat, outs = srv.replay(trace, arrival, keep_outputs=keep, timeout_ms=300000.0)
    info = srv.info()
    assert info["device_status"] == 0
    assert info["completed"] == n and info["in_flight"] == 0 and info["bytes_in_use"] == 0
    assert info["kernel_launches"] >= bursts
    assert np.all(np.isfinite(lat)) and np.all(lat > 0)
    for j in sorted(keep):
        k, op, Bj, _ = meta[j]
        s_, g_, _ = pool[meta[j]]
        for o, ref in zip(outs[j], _oracle(ROBOTS[k], op, s_, g_)):
            assert normwise(gen.from_soa(o, Bj), ref) < _tol(ROBOTS[k], op)
    srv.close()


def test_concurrent_submitters_and_collector(server):
    """Four threads submit at once (submit copies the inputs and publishes
    outside the server lock, one submitter at a time) while a fifth collects
    with wait_any: every request completes, its outputs are bit-identical to
    the same request served alone, and nothing stays in flight or reserved."""
    import threading

    srv, ids = server
    rng = np.random.default_rng(11)
    pool = []
    for j in range(12):
        k = j % len(ROBOTS)
        op = ["rnea", "crba", "aba", "rnea_grad"][j % 4]
        Bj = int(rng.integers(1, 300)) if ROBOTS[k].n_bodies < 64 else int(rng.integers(1, 64))
        _, _, inp = _inputs(ROBOTS[k], op, Bj, 2000 + j)
        alone, _ = _run(srv, ids[k], op, inp, Bj)
        pool.append((ids[k], op, Bj, inp, alone))
    n_threads, per_thread = 4, 120
    total = n_threads * per_thread
    owner = {}  # request -> pool index
    lock = threading.Lock()
    errors = []
    done = []

    def submitter(t):
        try:
            r = np.random.default_rng(100 + t)
            for _ in range(per_thread):
                p = int(r.integers(len(pool)))
                mid, op, Bj, inp, _ = pool[p]
                deadline = time.time() + 30.0
                while True:
                    req = srv.submit(mid, op, inp, Bj)
                    if req is not None:
                        break
                    assert time.time() < deadline, "server stayed busy"
                    time.sleep(1e-4)
                with lock:
                    owner[req] = p
        except Exception as e:  # reported by the main thread
            errors.append(e)

    def collector():
        try:
            deadline = time.time() + 60.0
            while len(done) < total:
                assert time.time() < deadline, "requests did not complete"
                try:
                    r = srv.wait_any(5.0)
                except fx.FraxError as e:
                    if e.status != 1:  # FRAX_EINVAL: nothing in flight yet
                        raise
                    time.sleep(1e-4)
                    continue
                if r is None:
                    continue
                with lock:
                    p = owner.get(r)
                if p is None:  # submitted, not yet recorded by its thread
                    time.sleep(1e-5)
                    continue
                mid, op, Bj, _, alone = pool[p]
                outs, _ = srv.collect(r, mid, op, Bj)
                done.append((p, outs))
        except Exception as e:
            errors.append(e)

    threads = [threading.Thread(target=submitter, args=(t,)) for t in range(n_threads)]
    col = threading.Thread(target=collector)
    col.start()
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    col.join()
    assert not errors, errors
    assert len(done) == total
    for p, outs in done:
        for a, b in zip(outs, pool[p][4]):
            assert np.array_equal(a, b)
    info = srv.info()
    assert info["in_flight"] == 0 and info["bytes_in_use"] == 0 and info["device_status"] == 0
