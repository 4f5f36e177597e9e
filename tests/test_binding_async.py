"""Host logic of the binding's asynchronous calls, on a stand-in for the
library (no device): the map holds every pending handle until the library
has finished it, since the library writes the call's results into the
handle's buffers as late as the map's destruction; results read back as the
synchronous call returns them."""
import ctypes
import gc
import weakref

import pytest

from paper_2603_03935_gb300 import binding as b


class FakeLib:
    """Queues calls as the library does and writes their results when the
    map's calls are finished (wait or destroy)."""

    def __init__(self, fail_frame=None):
        self.pending = []
        self.fail_frame = fail_frame
        self.destroyed = False

    def disc_integrate_frames_async(self, h, arr, n, stats, n_done, result):
        self.pending.append((stats, n_done, result, n))
        return 0

    def _finish(self):
        for stats, n_done, result, n in self.pending:
            done = n if self.fail_frame is None else min(n, self.fail_frame)
            for i in range(n):
                stats[i].valid_pixels = 100 + i
                stats[i].status = 0 if i < done else -7
            n_done._obj.value = done
            result._obj.value = 0 if done == n else -7
        self.pending = []
        return 0

    def disc_map_wait(self, h):
        return self._finish()

    def disc_map_destroy(self, h):
        self._finish()
        self.destroyed = True


@pytest.fixture
def fake_map(monkeypatch):
    """A DiscMap over a stand-in library; its handle is dropped at teardown,
    so a map a failed test left open never reaches the real library."""
    made = []

    def make(fake):
        monkeypatch.setattr(b, "lib", lambda: fake)
        m = b.DiscMap.__new__(b.DiscMap)
        m._h = b.c_vp(1)
        made.append(m)
        return m

    yield make
    for m in made:
        m._h = None


def test_pending_handles_live_until_the_map_finishes_them(fake_map):
    fake = FakeLib()
    m = fake_map(fake)
    h = m.integrate_frames_async([(b.Frame(), None)] * 3)
    ref = weakref.ref(h)
    del h
    gc.collect()
    h = ref()
    assert h is not None  # the map kept it: the library will still write into it
    assert m.wait() == 0
    stats, done, rc = h.result()
    assert (done, rc) == (3, 0) and [s["valid_pixels"] for s in stats] == [100, 101, 102]
    assert not m._pending  # released once finished
    m.close()
    assert fake.destroyed


def test_destroy_finishes_what_is_pending(fake_map):
    fake = FakeLib()
    m = fake_map(fake)
    h = m.integrate_frames_async([(b.Frame(), None)] * 2)
    m.close()
    assert fake.destroyed and h.done.value == 2 and h.rc.value == 0


def test_a_failed_call_raises_when_checked(fake_map):
    fake = FakeLib(fail_frame=1)
    m = fake_map(fake)
    h = m.integrate_frames_async([(b.Frame(), None)] * 4)
    with pytest.raises(b.DiscError):
        h.result()
    stats, done, rc = h.result(check=False)
    assert (done, rc) == (1, -7) and [s["status"] for s in stats] == [0, -7, -7, -7]
    m.close()


def test_raw_call_passes_the_callers_buffers(fake_map):
    fake = FakeLib()
    m = fake_map(fake)
    arr = (b.Frame * 2)()
    stats = (b.Stats * 2)()
    done, res = ctypes.c_int32(-1), ctypes.c_int32(1)
    assert m.integrate_frames_async_raw(arr, 2, stats, done, res) == 0
    assert (done.value, res.value) == (-1, 1)  # nothing written before the call is finished
    m.wait()
    assert (done.value, res.value) == (2, 0) and stats[1].valid_pixels == 101
    m.close()
