"""Host-side admission of the serving loop (no GPU): slots with workspace buffers kept across
requests, an HBM budget over those buffers, first come first served, and rejection of a request that
could never fit."""
from paper_2511_05233_gb300 import serve


def _reqs(sizes):
    return [serve.Request(rid=i, arrival=0.1 * i, side=8, porosity=0.5, corr_len=2.0, f_C=0.5, order=0)
            for i in range(len(sizes))], dict(enumerate(sizes))


def test_oversized_request_is_rejected_and_does_not_block_the_queue():
    reqs, size = _reqs([10, 500, 20, 30])
    adm = serve.Admission(slots=2, budget=100, size_of=lambda r: size[r.rid])
    accepted = [adm.arrive(r) for r in reqs]
    assert accepted == [True, False, True, True]
    assert reqs[1].result["status"].startswith("rejected")
    got = adm.admit()
    assert [r.rid for r, *_ in got] == [0, 2]               # two slots
    assert adm.admit() == []                                 # no slot free
    adm.release(got[0][2])
    nxt = adm.admit()
    assert [r.rid for r, *_ in nxt] == [3]
    assert adm.held() == 30 + 20                             # the freed slot's buffer grew from 10 to 30
    assert adm.idle()


def test_buffers_are_reused_and_the_budget_covers_them():
    reqs, size = _reqs([60, 30, 50])
    adm = serve.Admission(slots=2, budget=100, size_of=lambda r: size[r.rid])
    for r in reqs:
        adm.arrive(r)
    first = adm.admit()
    assert [(r.rid, slot, nbytes) for r, need, slot, nbytes in first] == [(0, 0, 60), (1, 1, 30)]
    assert adm.held() == 90
    # request 2 (50) would need slot 1's buffer grown to 50: 60 + 50 > 100, it waits
    assert adm.admit() == []
    adm.release(0)                                           # slot 0 holds 60 >= 50: reused as it is
    got = adm.admit()
    assert [(r.rid, slot, nbytes) for r, need, slot, nbytes in got] == [(2, 0, 60)]
    assert adm.held() == 90 and adm.idle()
