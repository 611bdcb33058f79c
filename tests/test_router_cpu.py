"""Host logic of the replica router (rfsr.Router) with fake engines and streams (no GPU):
placement by free memory budget, ties to the lowest engine index, and migration order (export,
import on the target, only then destroy the original, so a failed import leaves the stream where
it was)."""
import pytest

from paper_2203_09200_gb300 import rfsr


class FakeStream:
    def __init__(self, engine, tag):
        self.engine, self.tag, self.live = engine, tag, True

    def export_state(self):
        self.engine.log.append(("export", self.tag))
        return {"tag": self.tag}

    def destroy(self):
        self.engine.log.append(("destroy", self.tag))
        self.live = False


class FakeEngine:
    def __init__(self, budget, used, log, fail_import=False):
        self.budget, self.used, self.log, self.fail_import = budget, used, log, fail_import
        self.created = []

    def info(self):
        return {"memory_budget": self.budget, "memory_used": self.used}

    def create_stream(self, **kw):
        self.created.append(kw)
        return FakeStream(self, len(self.created))

    def import_stream(self, state):
        self.log.append(("import", state["tag"], id(self)))
        if self.fail_import:
            raise rfsr.RfsrError(rfsr.RFSR_ENOMEM, "no room")
        return FakeStream(self, state["tag"])


def test_place_most_free_budget():
    log = []
    e = [FakeEngine(8 << 30, 7 << 30, log), FakeEngine(8 << 30, 2 << 30, log),
         FakeEngine(4 << 30, 1 << 30, log)]
    r = rfsr.Router(e)
    assert r.place() is e[1]                    # 6 GB free against 1 and 3
    e[1].used = 6 << 30
    assert r.place() is e[2]                    # now 3 GB free against 1 and 2


def test_place_ties_go_to_lowest_index():
    log = []
    e = [FakeEngine(4 << 30, 1 << 30, log) for _ in range(3)]
    assert rfsr.Router(e).place() is e[0]
    e[0].used = 2 << 30
    assert rfsr.Router(e).place() is e[1]


def test_create_stream_forwards_arguments():
    log = []
    e = [FakeEngine(1 << 30, 0, log), FakeEngine(2 << 30, 0, log)]
    st = rfsr.Router(e).create_stream(height=720, width=1280, cc_mode="rme")
    assert st.engine is e[1] and e[1].created == [dict(height=720, width=1280, cc_mode="rme")]
    assert e[0].created == []


def test_migrate_order():
    log = []
    a, b = FakeEngine(1 << 30, 0, log), FakeEngine(1 << 30, 0, log)
    st = a.create_stream(height=64, width=64)
    moved = rfsr.Router([a, b]).migrate(st, b)
    assert moved.engine is b and moved.tag == st.tag
    assert log == [("export", st.tag), ("import", st.tag, id(b)), ("destroy", st.tag)]
    assert not st.live and moved.live


def test_failed_migration_keeps_the_original():
    log = []
    a, b = FakeEngine(1 << 30, 0, log), FakeEngine(1 << 30, 0, log, fail_import=True)
    st = a.create_stream(height=64, width=64)
    with pytest.raises(rfsr.RfsrError):
        rfsr.Router([a, b]).migrate(st, b)
    assert st.live and ("destroy", st.tag) not in log
