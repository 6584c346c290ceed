"""Host-side admission of the serving loop (no GPU): slots, HBM budget, first come first served,
and rejection of a request that could never fit."""
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
    got = [r.rid for r, _ in adm.admit()]
    assert got == [0, 2]                      # two slots
    assert adm.admit() == []                  # no slot free
    adm.release(10)
    assert [r.rid for r, _ in adm.admit()] == [3]
    assert adm.idle()


def test_budget_limits_admission_in_arrival_order():
    reqs, size = _reqs([60, 50, 10])
    adm = serve.Admission(slots=8, budget=100, size_of=lambda r: size[r.rid])
    for r in reqs:
        adm.arrive(r)
    # 60 fits, 50 does not fit next to it; the later 10 waits behind it (first come, first served)
    assert [r.rid for r, _ in adm.admit()] == [0]
    adm.release(60)
    assert [r.rid for r, _ in adm.admit()] == [1, 2]
