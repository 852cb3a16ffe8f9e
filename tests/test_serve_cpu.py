"""Host logic of the batching server: which waiting requests form a batch.

No device work: the admission rule only reads request sizes, kinds and keys."""
import numpy as np
import pytest

pytest.importorskip("torch")


def _req(rid, kind, n, eps_out=1.0, e0=(0.0, 0.0, 1.0)):
    from paper_1605_01715_gb300.serve import Request
    tri = np.zeros((n, 3, 3))
    sph = np.zeros((n, 4))
    extra = {}
    if kind == "polar":
        extra = dict(eps_in=np.full(n, 4.0), curv=np.ones(n), eps_out=eps_out, e0=e0)
    return Request(rid=rid, arrival=0.01 * rid, kind=kind, tri=tri, sph=sph, **extra)


def _server(**kw):
    from paper_1605_01715_gb300.serve import Server
    return Server(device="cpu", **kw)


def test_a_batch_takes_the_heads_kind_in_arrival_order():
    """Requests of the head's key join in arrival order; other kinds and other
    exterior permittivities or fields wait for a batch of their own."""
    srv = _server()
    w = [_req(0, "polar", 100), _req(1, "demag", 100), _req(2, "polar", 200), _req(3, "polar", 300, eps_out=2.0),
         _req(4, "polar", 400, e0=(1.0, 0.0, 0.0)), _req(5, "polar", 500)]
    group, need = srv._take_batch(w, 1 << 40, True)
    assert [r.rid for r in group] == [0, 2, 5]
    assert need == sum(srv._need(r) for r in group)
    group, _ = srv._take_batch(w[1:], 1 << 40, True)
    assert [r.rid for r in group] == [1]


def test_batch_limits_and_memory_budget():
    """At most max_batch requests and max_batch_points unknowns; within the memory left,
    except that the head is always admitted when nothing else is live."""
    srv = _server(max_batch=3, max_batch_points=1000)
    w = [_req(i, "demag", 300) for i in range(6)]
    group, _ = srv._take_batch(w, 1 << 40, True)
    assert [r.rid for r in group] == [0, 1, 2]          # max_batch
    srv = _server(max_batch=64, max_batch_points=700)
    group, _ = srv._take_batch(w, 1 << 40, True)
    assert [r.rid for r in group] == [0, 1]             # 900 > 700 unknowns
    one = srv._need(w[0])
    srv = _server()
    group, need = srv._take_batch(w, 2 * one + one // 2, False)
    assert [r.rid for r in group] == [0, 1] and need == 2 * one
    group, _ = srv._take_batch(w, one // 2, False)
    assert group == []                                   # nothing fits, something is live
    group, _ = srv._take_batch(w, one // 2, True)
    assert [r.rid for r in group] == [0]                 # nothing live: the head goes alone


def test_orders_per_kind():
    """The adjoint double layer of the polarization operator at p = 11 and the demag
    double layer at p = 10 by default; one p for both when given."""
    assert _server().p == {"polar": 11, "demag": 10}
    assert _server(p=8).p == {"polar": 8, "demag": 8}
    assert _server(p={"demag": 12}).p == {"polar": 11, "demag": 12}
