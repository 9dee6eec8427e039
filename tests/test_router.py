"""The replica router on the CPU: replicas are simulated by Python backends (a queue and a worker
thread each, serving at a set speed), so the routing policy -- scene placement, fewest outstanding
pixels, release on wait, error paths -- is checked without any GPU."""
import collections
import threading
import time

import pytest

import paper_2408_07967_gb300 as gs
from paper_2408_07967_gb300 import synth


class FakeReplicas:
    """Replica i finishes a request after pixels / speed[i] seconds of simulated work."""

    def __init__(self, speeds, fail_submit=()):
        self.speeds = list(speeds)
        self.fail_submit = set(fail_submit)
        self.lock = threading.Lock()
        self.next = 1
        self.done = {}
        self.got = collections.Counter()
        self.scenes = collections.defaultdict(set)
        self.queues = [collections.deque() for _ in speeds]
        self.cv = threading.Condition(self.lock)
        self.stop = False
        self.threads = [threading.Thread(target=self._work, args=(i,), daemon=True) for i in range(len(speeds))]
        for t in self.threads:
            t.start()

    def _work(self, i):
        while True:
            with self.cv:
                while not self.queues[i] and not self.stop:
                    self.cv.wait(0.01)
                if self.stop:
                    return
                ticket, px = self.queues[i].popleft()
            time.sleep(px / self.speeds[i])
            with self.cv:
                self.done[ticket] = True
                self.cv.notify_all()

    def submit(self, replica, scene, cam, opts, rgb, arrival):
        if replica in self.fail_submit:
            return -4, 0
        camd = gs._native.gs_camera.from_address(cam)
        with self.cv:
            t = self.next
            self.next += 1
            self.got[replica] += 1
            self.scenes[replica].add(scene)
            self.queues[replica].append((t, camd.width * camd.height))
            self.cv.notify_all()
        return 0, t

    def wait(self, replica, ticket, timeout_ms, out):
        deadline = time.time() + (timeout_ms / 1000.0 if timeout_ms >= 0 else 1e9)
        with self.cv:
            while ticket not in self.done:
                if time.time() >= deadline:
                    return -5
                self.cv.wait(0.005)
        out.status, out.batch_size, out.done_s, out.pairs = 0, 1, time.time(), replica
        return 0

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()


def cam(w, h):
    return synth.look_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), w, h)


def test_scene_placement_is_respected():
    fake = FakeReplicas([1e9] * 3)
    r = gs.Router(3, fake.submit, fake.wait)
    r.place_scene(0, 0)
    r.place_scene(0, 1)
    r.place_scene(1, 2)
    tickets = [r.submit(i % 2, cam(64, 64)) for i in range(40)]
    for t in tickets:
        _, rep = r.wait(t)
    assert fake.scenes[2] == {1} and 1 not in fake.scenes[0] | fake.scenes[1]
    assert fake.got[0] + fake.got[1] == 20 and fake.got[2] == 20
    with pytest.raises(gs.GsError):
        r.submit(7, cam(64, 64))                     # placed nowhere
    r.close()
    fake.close()


def test_fewest_outstanding_pixels():
    fake = FakeReplicas([1.0] * 3)                     # slow enough that nothing completes meanwhile
    r = gs.Router(3, fake.submit, fake.wait)
    for i in range(3):
        r.place_scene(0, i)
    t0 = r.submit(0, cam(3840, 2160))                  # 8.3 MP on replica 0
    assert r.outstanding(0) == (1, 3840 * 2160)
    small = [r.submit(0, cam(1280, 720)) for _ in range(18)]
    # the 0.92 MP requests fill replicas 1 and 2 first; replica 0 gets one only once they carry more
    got = [r.outstanding(i) for i in range(3)]
    assert got[0][0] == 1 and got[1][0] == 9 and got[2][0] == 9
    assert fake.got[1] == 9 and fake.got[2] == 9
    r.close()
    fake.close()


def test_waiting_releases_load_and_slow_replica_gets_less():
    fake = FakeReplicas([4e8, 4e8, 1e8])              # replica 2 is four times slower
    r = gs.Router(3, fake.submit, fake.wait)
    for i in range(3):
        r.place_scene(0, i)
    inflight = []
    reps = collections.Counter()

    def reap_one():                                     # the first request that has finished
        while True:
            for t in list(inflight):
                try:
                    _, rep = r.wait(t, 0)
                except gs.GsError:
                    continue
                inflight.remove(t)
                reps[rep] += 1
                return
            time.sleep(0.001)

    for i in range(120):                                # closed loop, 6 requests outstanding at most
        inflight.append(r.submit(0, cam(1920, 1080)))
        if len(inflight) >= 6:
            reap_one()
    while inflight:
        reap_one()
    assert sum(reps.values()) == 120
    assert reps[2] < reps[0] and reps[2] < reps[1]
    assert all(r.outstanding(i) == (0, 0) for i in range(3))
    r.close()
    fake.close()


def test_backend_errors_and_timeouts():
    fake = FakeReplicas([1.0, 1e9], fail_submit={0})
    r = gs.Router(2, fake.submit, fake.wait)
    r.place_scene(0, 0)
    with pytest.raises(gs.GsError):
        r.submit(0, cam(32, 32))                        # the only replica refuses: error, no load kept
    assert r.outstanding(0) == (0, 0)
    r.place_scene(1, 1)
    fake.speeds[1] = 32 * 32 / 0.3                      # 0.3 s of work
    t = r.submit(1, cam(32, 32))
    with pytest.raises(gs.GsError):
        r.wait(t, 10)                                   # still running: the ticket stays valid
    assert r.outstanding(1) == (1, 1024)
    st, rep = r.wait(t, 5000)
    assert st["status"] == 0 and rep == 1 and r.outstanding(1) == (0, 0)
    with pytest.raises(gs.GsError):
        r.wait(t)                                       # already waited for
    r.close()
    fake.close()


def test_concurrent_submits_spread_and_stay_consistent():
    fake = FakeReplicas([1e9] * 4)
    r = gs.Router(4, fake.submit, fake.wait)
    for i in range(4):
        r.place_scene(0, i)
    tickets = []
    lock = threading.Lock()

    def worker():
        mine = [r.submit(0, cam(100, 100)) for _ in range(50)]
        with lock:
            tickets.extend(mine)

    ths = [threading.Thread(target=worker) for _ in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert len(set(tickets)) == 200
    for t in tickets:
        r.wait(t)
    assert sum(fake.got.values()) == 200 and max(fake.got.values()) - min(fake.got.values()) <= 60
    assert all(r.outstanding(i) == (0, 0) for i in range(4))
    r.close()
    fake.close()


def test_bad_arguments():
    fake = FakeReplicas([1e9])
    with pytest.raises(gs.GsError):
        gs.Router(0, fake.submit, fake.wait)
    r = gs.Router(1, fake.submit, fake.wait)
    with pytest.raises(gs.GsError):
        r.place_scene(0, 1)                            # replica out of range
    with pytest.raises(gs.GsError):
        r.outstanding(3)
    r.close()
    fake.close()
