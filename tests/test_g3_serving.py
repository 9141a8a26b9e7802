"""Serving loop: continuous batching of frames through nam_submit/nam_poll.

Results equal a direct multi-material evaluation, are the same alone and in
a mix of concurrent frames, admission respects the HBM budget, and the
host-side failure paths (allocation failure, launch failure, a stalled
scheduler, cancellation, wait timeouts) end in a status, never a hang."""
import ctypes as C
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N_MAT = 4


@pytest.fixture(scope="module")
def scene():
    rng = W.rng_streams(77, 2 * N_MAT + 2)
    mats = []
    for k in range(N_MAT):
        pyr = W.make_pyramid(rng[k], 256, 256, 9, dtype=np.float16)
        model = W.make_model(rng[N_MAT + k], (14, 64, 64, 3), (8, 16, 6))
        mats.append((pyr, model))
    frames = []
    for (wd, ht) in ((320, 180), (256, 200), (640, 360)):
        q = W.warp_queries(rng[2 * N_MAT], wd, ht, 256, 256, order="tile")
        q.pop("xi")
        tiles = W.tile_ranges(wd, ht)
        mat_of_tile = rng[2 * N_MAT + 1].integers(0, N_MAT, len(tiles))
        frames.append((q, tiles, mat_of_tile))
    return mats, frames


def _ctx(**kw):
    from paper_2305_02678_gb300 import Context
    return Context(0, **kw)


def _materials(ctx, scene):
    return [ctx.material(256, 256, 9, p, m["frame"], m["decoder"]) for p, m in scene[0]]


class _Frame:
    """Host buffers of one submitted frame (kept alive until it completes)."""

    def __init__(self, B, q, tiles, mat_of_tile, mats, arrival=0.0):
        import torch
        self.q = {k: torch.from_numpy(v).pin_memory() for k, v in q.items()}
        self.n = len(q["u"])
        self.out = torch.full((self.n, 3), float("nan")).pin_memory()
        self.items = (B.nam_work_item * len(tiles))(*[B.nam_work_item(s, c, int(m)) for (s, c), m in
                                                      zip(tiles, mat_of_tile)])
        self.mat_arr = (C.c_void_p * len(mats))(*[m.h for m in mats])
        f = B.nam_frame()
        f.n_queries = self.n
        f.q = B.make_queries(self.q)
        f.items = C.addressof(self.items)
        f.n_items = len(tiles)
        f.n_materials = len(mats)
        f.materials = C.addressof(self.mat_arr)
        f.rgb_out = self.out.data_ptr()
        f.arrival_s = arrival
        self.f = f


def _direct(ctx, mats, q, tiles, mat_of_tile):
    import torch
    from paper_2305_02678_gb300 import binding as B
    dq = {k: torch.from_numpy(v).cuda() for k, v in q.items()}
    out = torch.zeros((len(q["u"]), 3), device="cuda")
    B.nam_eval_multi(ctx.h, [m.h for m in mats], dq, [(s, c, int(m)) for (s, c), m in zip(tiles, mat_of_tile)], out,
                     torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_frames_match_direct_evaluation_alone_and_in_a_mix(scene):
    from paper_2305_02678_gb300 import binding as B
    ctx = _ctx(serve_streams=4)
    mats = _materials(ctx, scene)
    q0, tiles0, m0 = scene[1][2]
    ref = _direct(ctx, mats, q0, tiles0, m0)
    # alone
    fr = _Frame(B, q0, tiles0, m0, mats)
    t = B.nam_submit(ctx.h, fr.f)
    st, stats = B.nam_wait(ctx.h, t, 30_000_000_000)
    assert st == 0 and stats.status == 0
    alone = fr.out.numpy().copy()
    assert np.array_equal(alone, ref)
    # in a mix: the same frame among 30 others of mixed size, submitted back to back
    keep, tickets = [], []
    target_idx = 17
    for i in range(31):
        q, tiles, mt = scene[1][i % 3] if i != target_idx else (q0, tiles0, m0)
        f = _Frame(B, q, tiles, mt, mats)
        keep.append(f)
        tickets.append(B.nam_submit(ctx.h, f.f))
    for t in tickets:
        st, _ = B.nam_wait(ctx.h, t, 60_000_000_000)
        assert st == 0
    assert np.array_equal(keep[target_idx].out.numpy(), alone)
    for i, f in enumerate(keep):
        q, tiles, mt = scene[1][i % 3] if i != target_idx else (q0, tiles0, m0)
        if i < 3:
            assert np.array_equal(f.out.numpy(), _direct(ctx, mats, q, tiles, mt))
    stats = ctx.stats()
    assert stats.completed == 32 and stats.failed == 0
    assert stats.p99_latency_ms >= stats.p50_latency_ms > 0
    ctx.close()


def test_served_frame_matches_the_oracle(scene, oracle):
    """One frame through nam_submit, every query checked against the FP64
    oracle of its tile's material (FP16 parameters, Sec. 5.2) at the FP16
    bound 2e-3 on the max, with the frame-conditioning band of the parity
    tests; the frame's recorded timeline is ordered."""
    from paper_2305_02678_gb300 import binding as B
    ctx = _ctx(serve_streams=2)
    mats = _materials(ctx, scene)
    q, tiles, mt = scene[1][0]
    fr = _Frame(B, q, tiles, mt, mats)
    t = B.nam_submit(ctx.h, fr.f)
    st, fs = B.nam_wait(ctx.h, t, 30_000_000_000)
    assert st == 0 and fs.status == 0
    g = fr.out.numpy().copy()
    ctx.close()
    n = len(q["u"])
    o = np.zeros((n, 3))
    kappa = np.zeros(n)
    gain = np.zeros((n, 3))
    for k, (pyr, model) in enumerate(scene[0]):
        idx = np.concatenate([np.arange(s, s + c) for (s, c), m in zip(tiles, mt) if m == k] or [np.zeros(0, int)])
        if len(idx) == 0:
            continue
        om = oracle.Model(256, 256, 9, pyr, model["frame"], model["decoder"], params="fp16")
        qk = {f: v[idx] for f, v in q.items()}
        o[idx] = oracle.eval(om, qk)
        kappa[idx] = oracle.frame_condition(om, qk)
        gain[idx] = oracle.band_gain(om, qk, kappa[idx])
    ok, s = oracle.parity(g, o, kappa, 2e-3, gain=gain)
    print(f"served frame {n} queries: max {s['max_rel']:.3e} (kappa <= 50: {s['max_rel_well_conditioned']:.3e}), "
          f"ill-conditioned {s['ill_conditioned']}")
    assert ok, s
    assert fs.submit_s <= fs.admit_s <= fs.start_s <= fs.enqueued_s <= fs.finish_s
    assert fs.slot in (0, 1) and fs.in_flight_at_admit == 0
    assert 0 < fs.gpu_begin_s <= fs.gpu_kernel_begin_s <= fs.gpu_kernel_end_s <= fs.gpu_end_s
    # device times sit on the host clock to within the anchor's error
    assert fs.start_s - 1e-3 <= fs.gpu_begin_s and fs.gpu_end_s <= fs.finish_s + 1e-3


def test_device_frame_needs_no_copies(scene):
    """NAM_FRAME_DEVICE: queries and RGB in device memory; the result is
    bitwise the direct evaluation, and the frame's device time from its first
    operation to its kernel holds only the work-table upload."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    ctx = _ctx(serve_streams=2)
    mats = _materials(ctx, scene)
    q, tiles, mt = scene[1][2]
    n = len(q["u"])
    dq = {k: torch.from_numpy(v).cuda() for k, v in q.items()}
    out = torch.full((n, 3), float("nan"), device="cuda")
    items = (B.nam_work_item * len(tiles))(*[B.nam_work_item(s, c, int(m)) for (s, c), m in zip(tiles, mt)])
    mat_arr = (C.c_void_p * len(mats))(*[m.h for m in mats])
    f = B.nam_frame()
    f.n_queries = n
    f.q = B.make_queries(dq)
    f.items = C.addressof(items)
    f.n_items = len(tiles)
    f.n_materials = len(mats)
    f.materials = C.addressof(mat_arr)
    f.rgb_out = out.data_ptr()
    f.flags = B.NAM_FRAME_DEVICE
    t = B.nam_submit(ctx.h, f)
    st, fs = B.nam_wait(ctx.h, t, 30_000_000_000)
    assert st == 0
    assert np.array_equal(out.cpu().numpy(), _direct(ctx, mats, q, tiles, mt))
    assert fs.gpu_kernel_begin_s - fs.gpu_begin_s < 2e-3
    ctx.close()


def test_future_arrival_is_held_until_then(scene):
    """A frame whose arrival time lies ahead waits in the queue until then."""
    from paper_2305_02678_gb300 import binding as B
    ctx = _ctx(serve_streams=2)
    mats = _materials(ctx, scene)
    q, tiles, mt = scene[1][1]
    arrival = B.nam_now() + 0.25
    fr = _Frame(B, q, tiles, mt, mats, arrival=arrival)
    t = B.nam_submit(ctx.h, fr.f)
    time.sleep(0.05)
    done, st = B.nam_poll(ctx.h, t)
    assert not done and ctx.stats().queued == 1
    st_code, fs = B.nam_wait(ctx.h, t, 30_000_000_000)
    assert st_code == 0
    assert fs.arrival_s == arrival and fs.admit_s >= arrival
    assert fs.admit_s - arrival < 0.05
    assert np.array_equal(fr.out.numpy(), _direct(ctx, mats, q, tiles, mt))
    ctx.close()


def test_frames_overlap_on_the_gpu(scene):
    """With several stream slots, a frame is admitted while another is still
    in flight (admission of frame k+1 precedes completion of frame k)."""
    from paper_2305_02678_gb300 import binding as B
    ctx = _ctx(serve_streams=4)
    mats = _materials(ctx, scene)
    q, tiles, mt = scene[1][2]
    frames = [_Frame(B, q, tiles, mt, mats) for _ in range(12)]
    tickets = [B.nam_submit(ctx.h, f.f) for f in frames]
    sts = [B.nam_wait(ctx.h, t, 60_000_000_000)[1] for t in tickets]
    overlapped = sum(1 for a, b in zip(sts, sts[1:]) if b.admit_s < a.finish_s)
    assert overlapped >= 1
    ctx.close()


def test_admission_respects_the_budget(scene):
    from paper_2305_02678_gb300 import binding as B
    q, tiles, mt = scene[1][2]
    n = len(q["u"])
    frame_bytes = n * 4 * 9 + n * 12
    ctx0 = _ctx()
    mats0 = _materials(ctx0, scene)
    mat_bytes = sum(m.info.resident_bytes for m in mats0)
    ctx0.close()
    # room for the materials and one frame at a time
    ctx = _ctx(hbm_budget_bytes=mat_bytes + int(frame_bytes * 1.5) + (1 << 20), serve_streams=4)
    mats = _materials(ctx, scene)
    frames = [_Frame(B, q, tiles, mt, mats) for _ in range(4)]
    tickets = [B.nam_submit(ctx.h, f.f) for f in frames]
    sts = [B.nam_wait(ctx.h, t, 60_000_000_000)[1] for t in tickets]
    for a, b in zip(sts, sts[1:]):
        assert b.admit_s >= a.finish_s - 1e-3   # one frame's buffers at a time
    assert all(s.status == 0 for s in sts)
    assert ctx.stats().resident_bytes <= ctx.stats().budget_bytes
    ctx.close()
    # a frame that can never fit is refused at submission
    ctx = _ctx(hbm_budget_bytes=mat_bytes + frame_bytes // 2)
    mats = _materials(ctx, scene)
    f = _Frame(B, q, tiles, mt, mats)
    with pytest.raises(B.NamError) as e:
        B.nam_submit(ctx.h, f.f)
    assert e.value.status == B.NAM_ERR_BUDGET
    ctx.close()


def test_failures_end_in_a_status(scene):
    from paper_2305_02678_gb300 import binding as B
    ctx = _ctx(serve_streams=2)
    mats = _materials(ctx, scene)
    q, tiles, mt = scene[1][0]
    # allocation failure of the frame's buffers
    B.nam_inject_fault(ctx.h, B.NAM_FAULT_ALLOC)
    f1 = _Frame(B, q, tiles, mt, mats)
    st, s = B.nam_wait(ctx.h, B.nam_submit(ctx.h, f1.f), 30_000_000_000)
    assert st == B.NAM_ERR_OOM and s.status == B.NAM_ERR_OOM
    # launch failure
    B.nam_inject_fault(ctx.h, B.NAM_FAULT_LAUNCH)
    f2 = _Frame(B, q, tiles, mt, mats)
    st, s = B.nam_wait(ctx.h, B.nam_submit(ctx.h, f2.f), 30_000_000_000)
    assert st == B.NAM_ERR_CUDA
    # a stalled scheduler: waits time out, queued frames can be cancelled
    B.nam_inject_fault(ctx.h, B.NAM_FAULT_STALL)
    f3 = _Frame(B, q, tiles, mt, mats)
    f4 = _Frame(B, q, tiles, mt, mats)
    t3 = B.nam_submit(ctx.h, f3.f)
    t4 = B.nam_submit(ctx.h, f4.f)
    st, _ = B.nam_wait(ctx.h, t3, 50_000_000)
    assert st == B.NAM_ERR_TIMEOUT
    done, _ = B.nam_poll(ctx.h, t3)
    assert not done
    assert B.nam_cancel(ctx.h, t4) == 0
    st, s = B.nam_wait(ctx.h, t4, 1_000_000_000)
    assert st == B.NAM_ERR_CANCELLED
    # recovery: the next frames run normally
    B.nam_inject_fault(ctx.h, B.NAM_FAULT_NONE)
    st, _ = B.nam_wait(ctx.h, t3, 30_000_000_000)
    assert st == 0
    assert np.isfinite(f3.out.numpy()).all()
    with pytest.raises(B.NamError) as e:
        B.nam_poll(ctx.h, 987654321)
    assert e.value.status == B.NAM_ERR_NOT_FOUND
    ctx.close()


def test_queue_depth_and_shutdown_with_pending_frames(scene):
    from paper_2305_02678_gb300 import binding as B
    ctx = _ctx(serve_streams=1, serve_queue_depth=3)
    mats = _materials(ctx, scene)
    q, tiles, mt = scene[1][0]
    B.nam_inject_fault(ctx.h, B.NAM_FAULT_STALL)
    keep = [_Frame(B, q, tiles, mt, mats) for _ in range(4)]
    for f in keep[:3]:
        B.nam_submit(ctx.h, f.f)
    with pytest.raises(B.NamError) as e:
        B.nam_submit(ctx.h, keep[3].f)
    assert e.value.status == B.NAM_ERR_BUSY
    t0 = time.time()
    ctx.close()   # cancels the queued frames, joins the scheduler
    assert time.time() - t0 < 10
