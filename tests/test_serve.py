"""Serving loop: admission and queueing logic on the CPU with fake maps and a fake
memory gauge; on the GPU, a mix of frames of different map sizes served concurrently,
each result bit-identical to the same frame run alone on a fresh map."""
import numpy as np
import pytest

from paper_2407_02363_b300 import serve


class FakeMap:
    def __init__(self, dims, log):
        self.dims, self.log, self.left = dims, log, 0

    def frame_host_async(self, cloud, chain, q, mask, centres, radii, out):
        self.left = 3                      # finishes on the third poll
        out[:] = cloud                     # "result" = the request's payload
        self.log.append(("launch", self.dims, cloud))

    def done(self):
        self.left -= 1
        return self.left <= 0


def _fake_server(free_total, budget=None, max_slots=8):
    log, state = [], {"free": free_total}

    def make_map(dims):
        state["free"] -= 100
        return FakeMap(dims, log)

    def release(m):
        state["free"] += 100
        log.append(("release", m.dims))

    srv = serve.Server(make_map=make_map, free_fn=lambda: state["free"], map_bytes=lambda d: 100,
                       link_mask=0, headroom=50, budget=budget, max_slots=max_slots,
                       alloc_out=lambda m: np.zeros(1), view_out=lambda b: b.copy(), release_map=release)
    return srv, log


def _reqs(sizes):
    return [serve.Request(rid=i, dims=(s, s, s), cloud=float(i), q=None, centres=None, radii=np.zeros(1),
                          arrival=0.0) for i, s in enumerate(sizes)]


def test_admission_by_free_memory_and_reuse():
    # room for exactly 2 slots: 340 free, 100 each, 50 headroom kept
    srv, log = _fake_server(free_total=340)
    done = srv.run(_reqs([128, 256, 128, 512, 256, 128]), realtime=False, poll_sleep=0, timeout=5)
    assert sorted(d.rid for d in done) == list(range(6))
    assert max(len(srv.slots), 0) <= 2                     # never more slots than memory allows
    assert srv.rejected_admissions > 0 and srv.evictions >= 1
    assert ("release", (128, 128, 128)) in log or ("release", (256, 256, 256)) in log
    launches = [e for e in log if e[0] == "launch"]
    assert len(launches) == 6


def test_every_request_completes_with_its_own_result_and_overlaps():
    srv, log = _fake_server(free_total=10_000)
    reqs = _reqs([128, 256, 512, 128, 256, 512, 128])
    done = srv.run(reqs, realtime=False, poll_sleep=0, timeout=5)
    assert sorted(d.rid for d in done) == list(range(7))
    for d in done:
        assert d.results[0] == float(d.rid)
    assert srv.max_inflight >= 3            # frames admitted while others were running
    assert len(srv.slots) <= 7


def test_budget_caps_slot_bytes():
    srv, _ = _fake_server(free_total=10_000, budget=250)
    done = srv.run(_reqs([128, 256, 512, 128]), realtime=False, poll_sleep=0, timeout=5)
    assert len(done) == 4
    assert srv.used_bytes() <= 250 and len(srv.slots) <= 2


@pytest.mark.gpu
def test_mixed_sizes_in_the_mix_equal_alone():
    from gpu_helpers import lib, spheres_bitequal
    v = lib()
    reqs, chains, spheres = serve.make_requests(7, 18, sizes=(128, 256), rate_hz=2000.0,
                                                points=(50_000, 400_000))
    srv = serve.gpu_server(chains, max_slots=6)
    done = srv.run(reqs, realtime=True, timeout=60)
    assert len(done) == len(reqs)
    assert srv.max_inflight >= 2
    by = {d.rid: d for d in done}
    alone_maps = {}
    for r in reqs:
        S = r.dims[0]
        if S not in alone_maps:
            m = v.Map(r.dims, 0.01)
            from paper_2407_02363_b300 import synth
            m.register_links(synth.link_models(chains[S], 0.01))
            alone_maps[S] = m
        ref = alone_maps[S].frame_host(r.cloud.numpy(), r.chain, r.q, 0b111, r.centres, r.radii)
        assert spheres_bitequal(by[r.rid].results, ref), r.rid
    for m in alone_maps.values():
        m.close()
    for s in srv.slots:
        s.map.close()
