"""The serving runtime: every served scan equals, bit for bit, the same scan
reconstructed directly with cbct_reconstruct (whose parity with the oracle the
reconstruction tests establish), whether it runs directly or as a graph
replay, in a fresh or a reused slot, under a tight arena that forces
evictions, and with one resident slot."""
import ctypes

import numpy as np
import pytest

from gpu_util import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1001_0599_gb300 import build, cbct
    build.build()
    cbct.load()
    assert torch.cuda.is_available()
    return cbct


def _scans(lib, names, n_each, seed=0):
    """(geometry, params, pinned sinogram) triples with seeded noisy inputs."""
    import torch
    from paper_1001_0599_gb300 import synthetic
    rng = np.random.default_rng(seed)
    out = []
    geoms = {}
    for name in names:
        wl = CASES[name] if name in CASES else synthetic.workload(name)
        geoms[name] = (wl, lib.geometry_from_workload(wl))
    tv = lib.TvParams.paper()
    for k in range(n_each):
        for name in names:
            wl, g = geoms[name]
            try:
                g.level_dims(1)
                levels = (3, 2)
            except lib.CbctError:
                levels = (4,)
            params = lib.make_recon_params(0.02, levels, tv, power_iters=10, clamp=True, power_iters_fine=2)
            truth = np.asarray(rng.random((wl.nx, wl.ny, wl.nz)), dtype=np.float32) * 0.02
            f = torch.from_numpy(truth).cuda()
            p = torch.empty(g.sino_shape, device="cuda")
            lib.cbct_forward_project(g, f, p)
            noisy = p + 0.01 * torch.randn(p.shape, device="cuda",
                                           generator=torch.Generator("cuda").manual_seed(seed * 1000 + k))
            out.append((name, g, params, noisy.cpu().contiguous().pin_memory()))
    return out


def _direct(lib, g, params, h_sino):
    import torch
    ws = lib.workspace(lib.cbct_workspace_size(g, params))
    st = lib.stats_buffer()
    vol = torch.zeros(g.vol_shape, device="cuda")
    lib.cbct_reconstruct(g, h_sino.cuda(), vol, params, ws, st)
    torch.cuda.synchronize()
    return vol.cpu().numpy(), lib.read_stats(st)


def _serve(lib, scans, **cfg):
    import torch
    srv = lib.Server(**cfg)
    outs = []
    tickets = []
    for name, g, params, h_sino in scans:
        h_vol = torch.empty(g.vol_shape).pin_memory()
        h_st = lib.pinned_stats_buffer()
        tickets.append(srv.submit(g, params, h_sino, h_vol, h_st))
        outs.append((h_vol, h_st))
    results = [srv.wait(t) for t in tickets]
    info = srv.query()
    srv.close()
    return [(v.numpy().copy(), lib.read_host_stats(s)) for v, s in outs], results, info


def test_served_scans_equal_direct_reconstruction(lib):
    scans = _scans(lib, ["small", "odd", "tall"], 2, seed=1)
    ref = [_direct(lib, g, p, s) for _, g, p, s in scans]
    for graphs in (True, False):
        got, res, info = _serve(lib, scans, use_graphs=graphs)
        assert info.completed == len(scans) and info.submitted == len(scans)
        for (v, st), (rv, rst), r in zip(got, ref, res):
            assert r.status == 0
            assert np.array_equal(v, rv)
            assert st.n_iters == rst.n_iters and st.flags == rst.flags
            assert list(st.tau[:2]) == list(rst.tau[:2])
            assert r.t_submit <= r.t_admit <= r.t_done and r.gpu_ms > 0
        if graphs:
            # one capture per slot: at least one slot per shape, at most one per scan
            assert 3 <= info.graphs_captured + info.graph_failures <= len(scans)
            if info.graph_failures == 0:
                # every scan runs as one launch of its slot's captured graph
                assert [r.graph_replay for r in res] == [1] * len(res)
        else:
            assert info.graphs_captured == 0 and all(r.graph_replay == 0 for r in res)


def test_tight_arena_evicts_and_one_slot_serialises(lib):
    scans = _scans(lib, ["small", "odd"], 3, seed=2)
    ref = [_direct(lib, g, p, s) for _, g, p, s in scans]
    sizes = []
    for _, g, p, _s in scans[:2]:
        sizes.append(lib.cbct_workspace_size(g, p) + 4 * (int(np.prod(g.sino_shape)) + int(np.prod(g.vol_shape))))
    arena = int(max(sizes) * 1.3) + (1 << 16)
    got, res, info = _serve(lib, scans, arena_bytes=arena, use_graphs=True)
    assert info.peak_bytes_in_use <= info.arena_bytes
    assert info.evictions > 0   # alternating shapes do not fit side by side
    for (v, _), (rv, _), r in zip(got, ref, res):
        assert r.status == 0 and np.array_equal(v, rv)
    got, res, info = _serve(lib, scans, max_resident=1, use_graphs=True)
    assert info.slots <= 1
    for (v, _), (rv, _), r in zip(got, ref, res):
        assert r.status == 0 and np.array_equal(v, rv)
    # arrival order is kept
    assert all(a.t_admit <= b.t_admit for a, b in zip(res, res[1:]))


def test_submit_validation(lib):
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl = CASES["small"]
    g = lib.geometry_from_workload(wl)
    params = lib.make_recon_params(0.02, (2,), lib.TvParams.paper())
    srv = lib.Server(arena_bytes=1 << 20)
    pinned_s = torch.zeros(g.sino_shape).pin_memory()
    pinned_v = torch.zeros(g.vol_shape).pin_memory()
    with pytest.raises(ValueError):   # pageable host buffers are refused by the binding
        srv.submit(g, params, torch.zeros(g.sino_shape), pinned_v)
    # and by the library itself
    t = ctypes.c_uint64()
    page = np.zeros(g.sino_shape, dtype=np.float32)
    st = lib.load().cbct_server_submit(srv.handle, g.handle, ctypes.byref(params), page.ctypes.data,
                                       pinned_v.data_ptr(), None, ctypes.byref(t))
    assert st == 1
    # a slot larger than the whole arena is refused up front
    with pytest.raises(lib.CbctError):
        srv.submit(g, params, pinned_s, pinned_v)
    with pytest.raises(lib.CbctError):
        srv.wait(12345)
    srv.close()
    # replay schedules are for parity tests, not for served scans
    srv = lib.Server()
    rp = lib.make_recon_params(0.02, (1,), lib.TvParams.paper(), taus=[1e-3], replay=[[1]])
    with pytest.raises(lib.CbctError):
        srv.submit(g, rp, pinned_s, pinned_v)
    srv.close()


def test_concurrent_submitters(lib):
    # four host threads submit and wait at once; every scan still equals its
    # direct reconstruction
    import threading

    import torch
    scans = _scans(lib, ["small", "odd"], 4, seed=3)
    ref = [_direct(lib, g, p, s) for _, g, p, s in scans]
    srv = lib.Server(use_graphs=True)
    outs = [None] * len(scans)
    errors = []

    def worker(k):
        try:
            for i in range(k, len(scans), 4):
                _, g, p, s = scans[i]
                h_vol = torch.empty(g.vol_shape).pin_memory()
                t = srv.submit(g, p, s, h_vol)
                r = srv.wait(t)
                outs[i] = (h_vol.numpy().copy(), r.status)
        except Exception as e:   # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    info = srv.query()
    srv.close()
    assert not errors
    assert info.completed == len(scans)
    for (v, status), (rv, _) in zip(outs, ref):
        assert status == 0 and np.array_equal(v, rv)


@pytest.mark.parametrize("lanes", [2, 3])
def test_concurrent_lanes_equal_direct_reconstruction(lib, lanes):
    # several reconstructions in flight on separate compute streams, each TV
    # solve on 1/lanes of the GPU: the solve's sums do not depend on its grid
    # size, so every scan still equals its direct reconstruction bit for bit
    scans = _scans(lib, ["small", "odd", "tall", "ragged_tma"], 2, seed=4)
    ref = [_direct(lib, g, p, s) for _, g, p, s in scans]
    for graphs in (True, False):
        got, res, info = _serve(lib, scans, use_graphs=graphs, concurrency=lanes)
        assert info.completed == len(scans)
        for (v, st), (rv, rst), r in zip(got, ref, res):
            assert r.status == 0
            assert np.array_equal(v, rv)
            assert st.n_iters == rst.n_iters and st.flags == rst.flags
            assert [st.iters[k].e_rof_last for k in range(st.n_iters)] == \
                [rst.iters[k].e_rof_last for k in range(rst.n_iters)]


def test_concurrency_validation(lib):
    with pytest.raises(lib.CbctError):
        lib.Server(concurrency=17)


def test_served_scan_matches_oracle(lib, orc):
    # a small scan served with concurrent lanes against the FP64 oracle run
    # on the served scan's own step decisions (its statistics), at 1e-4
    import torch
    from paper_1001_0599_gb300 import synthetic
    from gpu_util import TOL_RECON, f32, rel_l2
    wl = synthetic.workload("small")
    truth, y = synthetic.make_problem(wl)
    g = lib.geometry_from_workload(wl)
    p = orc.TVParams(eps_tv=1e-5)
    tv = lib.TvParams(p.eps_tv, p.c, p.alpha, p.rel_tol, p.max_inner, p.max_backtracks, p.s0)
    params = lib.make_recon_params(wl.lam, (6,), tv, power_iters=20)
    h_sino = torch.from_numpy(f32(y).astype(np.float32)).pin_memory()
    scans = [("small", g, params, h_sino)] * 3
    got, res, info = _serve(lib, scans, use_graphs=True, concurrency=3)
    og = orc.Geometry.from_workload(wl)
    for (v, st), r in zip(got, res):
        assert r.status == 0
        flat = list(st.steps[:st.n_steps])
        sched, k = [], 0
        for i in range(st.n_iters):
            n = int(st.iters[i].n_inner)
            sched.append(flat[k:k + n])
            k += n
        ref = orc.reconstruct(og, f32(y), wl.lam, (6,), p, power_iters=20, replay=sched)
        assert st.tau[0] == pytest.approx(ref.taus[0], rel=1e-5)
        assert rel_l2(v.astype(np.float64), ref.f) < TOL_RECON


@pytest.mark.parametrize("lanes", [1, 3])
def test_reused_steps_equal_direct_reconstruction(lib, lanes):
    # with reuse_steps, the first scan of each (geometry, parameters) pair runs
    # the power iterations and later scans of the pair take its taus: the
    # kernels are deterministic, so every scan still equals its direct
    # reconstruction bit for bit, with the same tau and L in its statistics
    import torch
    scans = _scans(lib, ["small", "odd", "tall"], 3, seed=5)
    ref = [_direct(lib, g, p, s) for _, g, p, s in scans]
    for graphs in (True, False):
        srv = lib.Server(use_graphs=graphs, concurrency=lanes, reuse_steps=True)
        got, res = [], []
        for batch in (scans[:3], scans[3:]):   # the second batch finds every pair's taus
            outs, tickets = [], []
            for name, g, params, h_sino in batch:
                h_vol = torch.empty(g.vol_shape).pin_memory()
                h_st = lib.pinned_stats_buffer()
                tickets.append(srv.submit(g, params, h_sino, h_vol, h_st))
                outs.append((h_vol, h_st))
            res += [srv.wait(t) for t in tickets]
            got += [(v.numpy().copy(), lib.read_host_stats(s)) for v, s in outs]
        info = srv.query()
        srv.close()
        assert [r.steps_reused for r in res] == [0] * 3 + [1] * 6
        assert info.step_reuses == 6 and info.completed == len(scans)
        for (v, st), (rv, rst), r in zip(got, ref, res):
            assert r.status == 0
            assert np.array_equal(v, rv)
            assert st.n_iters == rst.n_iters and st.flags == rst.flags
            assert list(st.tau[:2]) == list(rst.tau[:2])
            assert list(st.lipschitz[:2]) == list(rst.lipschitz[:2])


def test_serving_mix_shapes_equal_direct_reconstruction(lib):
    # two shapes of the serving mix at full size (128^3 at 2 mm with 20 views on
    # the 256x192 detector, 192x192x128 with 40 views on the 512x384 one), the
    # mix's 50-iteration 20/15/15 schedule, 2 lanes with step reuse: every
    # served scan, including those that reuse their shape's taus, equals its
    # direct reconstruction bit for bit
    import torch
    from paper_1001_0599_gb300 import synthetic
    shapes = [(128, 128, 128, 2.0, 2.0, 2.0, 256, 192, 1.56, 1.56, 20),
              (192, 192, 128, 4.0 / 3.0, 4.0 / 3.0, 1.0, 512, 384, 0.78, 0.78, 40)]
    tv = lib.TvParams.paper(eps_tv=1e-5)
    params = lib.make_recon_params(0.05, (20, 15, 15), tv, power_iters=20, clamp=True, power_iters_fine=4)
    scans = []
    for k, (nx, ny, nz, dx, dy, dz, nu, nv, du, dv, views) in enumerate(shapes):
        wl = synthetic.Workload(f"mix{k}", nx, ny, nz, dx, dy, dz, nu, nv, du, dv, views, photons=5e4,
                                phantom="head_neck", phantom_seed=3, noise_seed=10, lam=0.05, iters=(20, 15, 15))
        g = lib.geometry_from_workload(wl)
        truth = synthetic.voxelise(synthetic.make_phantom(wl), nx, ny, nz, dx, dy, dz).astype(np.float32)
        p = torch.empty(g.sino_shape, device="cuda")
        lib.cbct_forward_project(g, torch.from_numpy(truth).cuda(), p)
        for rep in range(2):
            gen = torch.Generator(device="cuda").manual_seed(100 * k + rep)
            counts = torch.poisson(wl.photons * torch.exp(-p), generator=gen)
            y = torch.log(wl.photons / counts.clamp_min(1.0)).float()
            scans.append((wl.name, g, params, y.cpu().contiguous().pin_memory()))
    ref = [_direct(lib, g, p, s) for _, g, p, s in scans]
    srv = lib.Server(use_graphs=True, concurrency=2, reuse_steps=True)
    got, res = [], []
    for batch in (scans[0::2], scans[1::2]):   # the second scan of each shape reuses the first one's taus
        outs, tickets = [], []
        for name, g, p, h_sino in batch:
            h_vol = torch.empty(g.vol_shape).pin_memory()
            h_st = lib.pinned_stats_buffer()
            tickets.append(srv.submit(g, p, h_sino, h_vol, h_st))
            outs.append((h_vol, h_st))
        res += [srv.wait(t) for t in tickets]
        got += [(v.numpy().copy(), lib.read_host_stats(s)) for v, s in outs]
    srv.close()
    ref = [ref[i] for i in (0, 2, 1, 3)]
    assert [r.steps_reused for r in res] == [0, 0, 1, 1]
    for (v, st), (rv, rst), r in zip(got, ref, res):
        assert r.status == 0
        assert np.array_equal(v, rv)
        assert list(st.tau[:3]) == list(rst.tau[:3]) and list(st.lipschitz[:3]) == list(rst.lipschitz[:3])
