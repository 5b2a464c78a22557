"""Host logic of the continuous-batching server that needs no GPU: how a
batch is taken from one (operation, n) queue.  A key with at least HOT
waiting requests is served alone (a single-key call, which can take the
tensor-core product); a batch whose requests all share one key is also a
single-key call (a lone request at low load takes the plain per-request
call); otherwise the oldest requests across keys form a multi-key batch;
KeyGen requests never wait for a key; per-request mode always takes one."""
import collections

from paper_2606_01211_gb300 import serve


class _Cfg:
    plain = False


def _engine(plain=False):
    eng = serve.Engine.__new__(serve.Engine)  # the queue logic only: no device state
    eng.cfg = _Cfg()
    eng.cfg.plain = plain
    return eng


def _queue(keys, op=1):
    fifo = collections.deque(serve.Request(i, op, 976, k, float(i)) for i, k in enumerate(keys))
    per_key = collections.Counter(keys)
    return fifo, per_key


def test_hot_key_is_served_alone_in_arrival_order():
    eng = _engine()
    keys = [7] * eng.HOT + [1, 2, 3]
    keys[3], keys[-1] = 2, 7  # interleave
    fifo, per_key = _queue(keys)
    group, single = eng._take(fifo, per_key, mb=512)
    assert single and {q.key for q in group} == {7}
    assert [q.rid for q in group] == sorted(q.rid for q in group)
    assert len(group) == keys.count(7)
    assert per_key[7] == 0
    assert sorted(q.key for q in fifo) == sorted(k for k in keys if k != 7)


def test_mixed_keys_below_the_threshold_form_a_multi_key_batch():
    eng = _engine()
    fifo, per_key = _queue([1, 2, 1, 3, 2])
    group, single = eng._take(fifo, per_key, mb=4)
    assert not single and [q.rid for q in group] == [0, 1, 2, 3]
    assert len(fifo) == 1 and per_key == collections.Counter({2: 1, 1: 0, 3: 0})


def test_one_key_batch_is_a_single_key_call():
    eng = _engine()
    fifo, per_key = _queue([5, 5, 5])
    group, single = eng._take(fifo, per_key, mb=512)
    assert single and len(group) == 3 and not fifo


def test_keygen_requests_are_taken_in_order_and_per_request_mode_takes_one():
    eng = _engine()
    fifo, per_key = _queue([-1] * 100, op=0)
    group, _ = eng._take(fifo, per_key, mb=64)
    assert [q.rid for q in group] == list(range(64))
    plain = _engine(plain=True)
    fifo, per_key = _queue([4] * 100)
    group, single = plain._take(fifo, per_key, mb=1)
    assert len(group) == 1 and single
