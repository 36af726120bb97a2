"""Failure handling without faulting the GPU: an HBM budget that a request
exceeds (CAT_ENOMEM, the context stays usable and returns its memory), the
server admitting a request larger than a worker's share (that ticket fails,
the next succeeds), and waits that time out on the host."""
import pytest

from paper_2601_11621_gb300 import capi

pytestmark = pytest.mark.gpu


def test_context_budget_enomem_and_recovery(orc, cat_lib):
    c = capi.Context(0, hbm_budget_bytes=4 << 20)  # 4 MiB of scratch
    try:
        with pytest.raises(capi.CatError) as e:
            capi.catalan_exact(c, 10**7)
        assert e.value.code == capi.CAT_ENOMEM
        in_use, _ = c.memory()
        assert in_use == 0  # everything taken before the failure was returned
        r = capi.to_numpy(capi.catalan_exact(c, 5000))
        assert (r == orc.catalan(5000)).all()
        assert c.memory()[0] == 0
    finally:
        c.close()


def test_server_denies_oversized_request_then_serves(orc, cat_lib):
    from paper_2601_11621_gb300.server import Server
    sv = Server(0, hbm_budget_bytes=32 << 20, workers=1, max_batch=16)
    try:
        with pytest.raises(capi.CatError) as e:
            sv.submit(0, 2 * 10**7)   # estimate 1.25 M limbs x 256 B, far above 32 MiB
        assert e.value.code == capi.CAT_ENOMEM
        assert sv.pending() == (0, 0)
        small = sv.submit(0, 777)
        got = sv.fetch_host(small)
        assert (got == orc.catalan(777)).all()
        assert sv.release(small) == 0
    finally:
        sv.close()


def test_server_wait_timeout_is_a_host_status(orc, cat_lib):
    from paper_2601_11621_gb300.server import Server
    sv = Server(0, hbm_budget_bytes=8 * 10**9, workers=1, max_batch=16)
    try:
        t = sv.submit(0, 2 * 10**8)      # tens of milliseconds of work
        try:
            sv.wait(t, timeout_ms=0)
            timed_out = False
        except capi.CatError as e:
            assert e.code == capi.CAT_ETIMEOUT
            timed_out = True
        r = sv.wait(t)                   # the request itself completes normally
        assert r.length > 0
        assert timed_out  # a zero timeout cannot outlast tens of milliseconds of work
        assert sv.release(t) == 0
    finally:
        sv.close()
