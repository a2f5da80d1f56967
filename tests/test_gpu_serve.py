"""Serving loop (ssgi_serve_*): each result is the same alone and in a concurrent mix, and
admission, budget, queue, bounded waits and cancellation behave as the header states.
Failures are made on the host (oversized or malformed requests, a blocked queue); nothing here
faults or hangs the GPU, and every wait has a timeout."""
import numpy as np
import pytest
import torch

import ssgi_inputs as si

pytestmark = pytest.mark.gpu


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _direct(S, wl):
    """The same request through the per-call C ABI on the current stream."""
    g, env, cams, _ = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    lut = S.ssgi_build_brdf_lut()
    em = S.ssgi_build_env_mips(env)
    hiz = S.ssgi_build_hiz(g.depth, p.hiz_levels) if p.hiz_levels > 1 else None
    c_d, _, c1 = S.ssgi_shade_direct(g, cams, em, lut)
    tr = S.ssgi_trace_indirect(g, cams, hiz, c1, c_d, em, p)
    torch.cuda.synchronize()
    return tr["final"].cpu().numpy()


def _requests():
    out = []
    for i, (H, W, spp, steps) in enumerate([(48, 64, 4, 32), (75, 131, 8, 48), (90, 160, 16, 64), (37, 53, 7, 20),
                                            (64, 64, 32, 64), (120, 200, 4, 64)]):
        wl = si.small_case(seed=40 + i, H=H, W=W, spp=spp, env_hw=(32, 64) if i % 2 else (16, 32), max_steps=steps)
        out.append(wl)
    return out


def _submit(srv, S, wl, out, scene=-1):
    p = S.params_of(wl.params)
    if scene >= 0:
        return srv.submit(out, _pinned(wl.env), p, scene=scene)
    return srv.submit(out, _pinned(wl.env), p, depth=_pinned(wl.depth), normal=_pinned(wl.normal),
                      albedo=_pinned(wl.albedo), rough=_pinned(wl.rough), metal=_pinned(wl.metal), cams=wl.cams)


def test_results_are_identical_alone_and_in_a_mix():
    import paper_2504_01358_gb300 as S
    from paper_2504_01358_gb300 import _native as N
    from paper_2504_01358_gb300.serve import Server

    reqs = _requests()
    ref = [_direct(S, wl) for wl in reqs]
    # alone: one slot, one request at a time
    alone = []
    with Server(256 << 20, max_slots=1, queue_capacity=4) as srv:
        for wl in reqs:
            out = torch.zeros(tuple(wl.depth.shape) + (3,)).pin_memory()
            rc, t = _submit(srv, S, wl, out)
            assert rc == N.OK
            rc, lat = srv.wait(t, 30000)
            assert rc == N.OK and lat > 0
            alone.append(out.numpy().copy())
    # mix: four slots, everything submitted at once, two requests on a resident scene
    with Server(256 << 20, max_slots=4, queue_capacity=64) as srv:
        sid = srv.scene_add(_pinned(reqs[2].depth), _pinned(reqs[2].normal), _pinned(reqs[2].albedo),
                            _pinned(reqs[2].rough), _pinned(reqs[2].metal), reqs[2].cams, reqs[2].params.hiz_levels)
        outs, tickets = [], []
        for k in range(3):
            for i, wl in enumerate(reqs):
                out = torch.zeros(tuple(wl.depth.shape) + (3,)).pin_memory()
                rc, t = _submit(srv, S, wl, out, scene=sid if (i == 2 and k == 1) else -1)
                assert rc == N.OK
                outs.append((i, out))
                tickets.append(t)
        for t in tickets:
            rc, _ = srv.wait(t, 60000)
            assert rc == N.OK
        st = srv.stats()
        assert st["completed"] == len(tickets) and st["in_flight"] == 0 and st["queued"] == 0
        assert srv.scene_remove(sid) == N.OK
    for i, out in outs:
        assert np.array_equal(out.numpy(), alone[i]), i
    for i in range(len(reqs)):
        assert np.array_equal(alone[i], ref[i]), i


def test_admission_waits_for_memory_and_slots():
    import paper_2504_01358_gb300 as S
    from paper_2504_01358_gb300 import _native as N
    from paper_2504_01358_gb300.serve import Server, ssgi_serve_request_bytes

    wl = si.small_case(seed=3, H=120, W=200, spp=8)
    need = ssgi_serve_request_bytes(wl.depth.shape, 16, 32, 8, False)
    budget = max(2 * need + need // 2, 1 << 20)  # room for two requests at a time
    with Server(budget, max_slots=4, queue_capacity=16) as srv:
        outs, tickets = [], []
        for _ in range(6):
            out = torch.zeros(tuple(wl.depth.shape) + (3,)).pin_memory()
            rc, t = _submit(srv, S, wl, out)
            assert rc == N.OK
            outs.append(out)
            tickets.append(t)
        for t in tickets:
            assert srv.wait(t, 60000)[0] == N.OK
        st = srv.stats()
        assert st["arena_bytes_peak"] <= budget
        assert st["completed"] == 6
    for o in outs[1:]:
        assert np.array_equal(o.numpy(), outs[0].numpy())


def test_rejections_timeouts_and_cancellation():
    import paper_2504_01358_gb300 as S
    from paper_2504_01358_gb300 import _native as N
    from paper_2504_01358_gb300.serve import Server, ssgi_serve_request_bytes

    big = si.small_case(seed=9, H=200, W=300, spp=4)
    small = si.small_case(seed=8, H=48, W=64, spp=4)
    need_small = ssgi_serve_request_bytes(small.depth.shape, 16, 32, 8, False)
    budget = 4 << 20
    assert ssgi_serve_request_bytes(big.depth.shape, 16, 32, 8, False) > budget
    with Server(budget, max_slots=2, queue_capacity=2) as srv:
        out_big = torch.zeros(tuple(big.depth.shape) + (3,)).pin_memory()
        assert _submit(srv, S, big, out_big)[0] == N.BUDGET  # alone larger than the arena
        bad_env = np.ones((3, 8, 3), np.float32)
        out = torch.zeros(tuple(small.depth.shape) + (3,)).pin_memory()
        rc, _ = srv.submit(out, bad_env, S.params_of(small.params), depth=small.depth, normal=small.normal,
                           albedo=small.albedo, rough=small.rough, metal=small.metal, cams=small.cams)
        assert rc == N.INVALID_ARG
        # fill the arena with a resident scene so that the next request cannot be admitted
        filler = None
        for h in range(16, 600, 4):  # a scene that leaves less than one small request of room
            shape = (1, h, h)
            scene_bytes = (ssgi_serve_request_bytes(shape, 16, 32, 8, False) -
                           ssgi_serve_request_bytes(shape, 16, 32, 8, True))
            if budget - need_small < scene_bytes <= budget:
                filler = si.small_case(seed=1, H=h, W=h, spp=1)
                break
        assert filler is not None
        sid = srv.scene_add(filler.depth, filler.normal, filler.albedo, filler.rough, filler.metal, filler.cams, 8)
        rc, t1 = _submit(srv, S, small, out)
        assert rc == N.OK
        out2 = torch.zeros_like(out).pin_memory()
        rc, t2 = _submit(srv, S, small, out2)
        assert rc == N.OK
        out3 = torch.zeros_like(out).pin_memory()
        assert _submit(srv, S, small, out3)[0] == N.QUEUE_FULL  # two already wait
        assert srv.wait(t1, 100)[0] == N.TIMEOUT  # cannot be admitted while the scene holds the arena
        assert srv.poll(t1)[0] == N.NOT_READY
        assert srv.cancel(t1) == N.OK
        assert srv.poll(t1)[0] == N.CANCELLED
        assert srv.poll(t1)[0] == N.INVALID_ARG  # collected
        assert srv.scene_remove(sid) == N.OK  # frees the arena: t2 is admitted and finishes
        assert srv.wait(t2, 30000)[0] == N.OK
        st = srv.stats()
        assert st["cancelled"] == 1 and st["rejected"] >= 3 and st["completed"] == 1
    assert np.array_equal(out2.numpy(), _direct(S, small))


def test_destroy_cancels_queued_requests():
    import paper_2504_01358_gb300 as S
    from paper_2504_01358_gb300 import _native as N
    from paper_2504_01358_gb300.serve import Server

    wl = si.small_case(seed=12, H=90, W=160, spp=32, max_steps=64)
    srv = Server(64 << 20, max_slots=1, queue_capacity=64)
    outs = []
    for _ in range(12):
        out = torch.zeros(tuple(wl.depth.shape) + (3,)).pin_memory()
        assert _submit(srv, S, wl, out)[0] == N.OK
        outs.append(out)
    assert srv.close(timeout_ms=60000) == N.OK
