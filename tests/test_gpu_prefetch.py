"""GPU checks of the learned prefetcher: network gradients and Adam step
against the FP64 oracle (bf16 tolerance), learning on a synthetic task, the
device-built network input and targets, prefetch placement bit-exact
against the oracle's sequential definition, and the miss reduction on
abrupt-turn trajectories."""
import math

import numpy as np
import pytest

import oracle
import scenegen
from _common import import_scene
from oracle import build as ob
from oracle import mlp as om
from oracle import residency as rs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_19415_b300 as mod
    return mod


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _maxdev(a, b):
    """Largest element-wise deviation relative to the reference's largest magnitude."""
    b = np.asarray(b, np.float64)
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("shape", [(28, 64, 256, 32), (12 + 256, 256, 4096, 256), (20, 48, 80, 7)])
def test_gradients_match_oracle(v, shape):
    import torch
    I, H, O, B = shape
    p = v.Prefetcher(v.MlpShape(n_in=I, n_hidden=H, n_out=O, max_batch=max(B, 8), seed=3, lr=0.0))
    rng = np.random.default_rng(I + O)
    P = {"W1": rng.normal(0, 1 / math.sqrt(I), (I, H)), "b1": rng.normal(0, 0.1, H),
         "W2": rng.normal(0, 1 / math.sqrt(H), (H, H)), "b2": rng.normal(0, 0.1, H),
         "W3": rng.normal(0, 1 / math.sqrt(H), (H, O)), "b3": rng.normal(0, 0.1, O)}
    p.set_params({k: a.astype(np.float32) for k, a in P.items()})
    x = rng.normal(0, 1, (B, I)).astype(np.float32)
    y = (rng.random((B, O)) < 0.2).astype(np.float32)
    m = (rng.random((B, O)) < 0.9).astype(np.float32)
    dev = "cuda"
    X, Yt, Mt = (torch.from_numpy(a).to(dev) for a in (x, y, m))
    loss = torch.zeros(1, device=dev)
    p.train_step(X, Yt, Mt, loss_out=loss)
    g = p.grads()
    # oracle on the bf16-rounded weights and input the tensor cores see
    Wb = {k: (om.bf16_round(a.astype(np.float32)) if k.startswith("W") else a.astype(np.float32).astype(np.float64))
          for k, a in P.items()}
    ref_loss, ref_g, _ = om.loss_and_grads(Wb, om.bf16_round(x), y.astype(np.float64), m.astype(np.float64))
    assert abs(float(loss.item()) - ref_loss) < 1e-2 * max(1.0, abs(ref_loss))
    # (norm-relative: the GPU's hidden activations and backward signals are
    # bf16, so a ReLU whose pre-activation lies within bf16 rounding of 0
    # may take the other derivative than in the FP64 oracle, which moves
    # single gradient elements by several percent of the tensor's largest)
    for k in ref_g:
        assert _rel(g[k], ref_g[k]) < 3e-2, (k, _rel(g[k], ref_g[k]))
    # the forward pass is continuous in those roundings, so its logits are
    # also held element by element: each bf16 rounding is at most 2^-9
    # relative, and a sum of products of mixed signs keeps its error near
    # 2^-9 of its size, so 5% of the largest logit is a wide margin
    logits = p.forward(X).cpu().numpy()
    ref = om.forward(Wb, om.bf16_round(x))["logits"]
    assert _rel(logits, ref) < 2e-2 and _maxdev(logits, ref) < 5e-2
    # batch 1 (the inference GEMV, not the tensor-core GEMM)
    one = p.forward(X[:1]).cpu().numpy()
    assert _rel(one, ref[:1]) < 2e-2 and _maxdev(one, ref[:1]) < 5e-2


def test_adam_step_matches_oracle(v):
    import torch
    I, H, O, B = 28, 64, 128, 16
    p = v.Prefetcher(v.MlpShape(n_in=I, n_hidden=H, n_out=O, max_batch=B, seed=9, lr=1e-3))
    P0 = p.params()
    rng = np.random.default_rng(1)
    x = rng.normal(0, 1, (B, I)).astype(np.float32)
    y = (rng.random((B, O)) < 0.3).astype(np.float32)
    m = np.ones((B, O), np.float32)
    p.train_step(*(torch.from_numpy(a).cuda() for a in (x, y, m)))
    g = p.grads()
    P1 = p.params()
    zeros = {k: np.zeros_like(a, np.float64) for k, a in P0.items()}
    ref, _, _ = om.adam({k: a.astype(np.float64) for k, a in P0.items()},
                        {k: a.astype(np.float64) for k, a in g.items()}, zeros, zeros, 1, lr=1e-3)
    for k in P0:
        np.testing.assert_allclose(P1[k], ref[k], rtol=1e-5, atol=1e-6)


def test_network_learns(v):
    """A learnable target (page j wanted iff x . u_j > 0) drives the loss down."""
    import torch
    I, H, O, B = 28, 64, 256, 128
    p = v.Prefetcher(v.MlpShape(n_in=I, n_hidden=H, n_out=O, max_batch=B, seed=2, lr=3e-3))
    rng = np.random.default_rng(0)
    U = rng.normal(size=(I, O))
    X = rng.normal(size=(4096, I)).astype(np.float32)
    Y = (X @ U > 0).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    Md = torch.ones_like(Yd)
    from paper_2506_19415_b300 import prefetch_train as pt
    curve = pt.train(p, Xd, Yd, Md, steps=400, batch=B)
    assert curve[-1] < 0.5 * curve[0], curve


def _blob_scene():
    raw = scenegen.blob_scene(n=120_000, n_blobs=40, lo=0.0, hi=40.0, sh_degree=1, seed=44)
    bp = ob.BuildParams(page_size=512, paging="octree", lo=(-5, -5, -5), hi=(45, 45, 45), voxel=50 / 40, kappa=1.0,
                        link_samples=2)
    return raw, ob.build_scene(raw, bp)


def test_features_and_labels(v):
    import torch
    raw, sc = _blob_scene()
    scene = import_scene(v, raw, sc)
    n_out = 64
    r = v.Renderer(scene, v.RenderConfig(max_width=320, max_height=180, lod=False), pool_slots=8)
    cams = scenegen.random_fly_path(3, seed=7, lo=0.0, hi=40.0, width=320, height_px=180, speed=1.0)
    r.render_feedback([cams[1]])
    x = torch.empty(12 + n_out // 16, device="cuda")
    base = torch.empty(1, dtype=torch.int32, device="cuda")
    v.vm3dgs_prefetch_features(r, n_out, cams[1], cams[0], x, base)
    y = torch.empty(n_out, device="cuda")
    m = torch.empty(n_out, device="cuda")
    v.vm3dgs_prefetch_labels(r, n_out, base, y, m)
    req = r.debug(v.DBG_REQ, np.uint32)
    # accumulated labels: the OR with what y already holds
    y2 = torch.zeros(n_out, device="cuda")
    y2[::3] = 1.0
    v.vm3dgs_prefetch_labels(r, n_out, base, y2, m, accumulate=True)
    cen = rs.page_centroids(sc)
    pos = cams[1].campos.astype(np.float32)
    d2 = ((cen[:, :3] - pos) ** 2).sum(1)
    pstar = int(np.argmin(d2))
    b = min(max(pstar - n_out // 2, 0), max(sc.n_pages - n_out, 0))
    assert int(base.item()) == b
    lo, hi = cen[:, :3].min(0).astype(np.float64), cen[:, :3].max(0).astype(np.float64)
    c, half = 0.5 * (lo + hi), max(0.5 * (hi - lo))
    f, g = cams[1].view[2, :3], cams[0].view[2, :3]
    want = np.concatenate([(pos - c) / half, f, (pos - cams[0].campos) / (0.01 * half), (f - g) * 10.0])
    np.testing.assert_allclose(x.cpu().numpy()[:12], want, rtol=1e-4, atol=1e-5)
    hist = [sum(1 for k in range(16) if b + 16 * i + k < sc.n_pages and req[b + 16 * i + k]) / 16 for i in range(n_out // 16)]
    np.testing.assert_array_equal(x.cpu().numpy()[12:], np.float32(hist))
    yy = np.array([1.0 if b + j < sc.n_pages and req[b + j] else 0.0 for j in range(n_out)], np.float32)
    np.testing.assert_array_equal(y.cpu().numpy(), yy)
    want2 = yy.copy()
    want2[::3] = 1.0
    np.testing.assert_array_equal(y2.cpu().numpy(), want2)
    np.testing.assert_array_equal(m.cpu().numpy(), (b + np.arange(n_out) < sc.n_pages).astype(np.float32))


def test_prefetch_placement_parity(v):
    """Fixed logits (network output = bias) so both sides see the same scores:
    after every frame's feedback-driven update and prefetch, the page table and
    the prefetch copy list equal the oracle's, and the pool holds the pages."""
    raw, sc = _blob_scene()
    scene = import_scene(v, raw, sc)
    n_out = 128
    W, H = 320, 180
    P = 10
    rec = scene.info.record_bytes
    budget = 4 * 512 * rec
    r = v.Renderer(scene, v.RenderConfig(max_width=W, max_height=H, lod=False, staging_bytes=budget), pool_slots=P)
    p = v.Prefetcher(v.MlpShape(n_in=12 + n_out // 16, n_hidden=32, n_out=n_out, max_batch=1, seed=1, lr=0.0))
    rng = np.random.default_rng(5)
    b3 = rng.permutation(n_out).astype(np.float32) / n_out - 0.3   # distinct scores, ~30% below 0
    Pp = p.params()
    Pp["W3"][:] = 0
    Pp["b3"][:] = b3
    p.set_params(Pp)
    rp = rs.ResidencyParams(n_entries=P, page_size=512, levels=1, fanout=8, record_bytes=rec, budget_bytes=budget,
                            lod=False)
    pt = rs.PageTable(rp)
    cen = rs.page_centroids(sc)
    cams = scenegen.random_fly_path(8, seed=3, lo=0.0, hi=40.0, width=W, height_px=H, speed=2.0)
    host = scene.pages(0)
    for t, cam in enumerate(cams):
        prev = cams[t - 1] if t else cam
        r.render_feedback([cam])
        r.update_residency()
        v.vm3dgs_prefetch(r, p, cam, prev, 0.0)
        ref = oracle.frame(sc, pt, cam, ds=4, render_image=False)
        d2 = ((cen[:, :3] - cam.campos.astype(np.float32)) ** 2).sum(1)
        base = min(max(int(np.argmin(d2)) - n_out // 2, 0), max(sc.n_pages - n_out, 0))
        copies = rs.prefetch(pt, b3, base, 0.0, ref["req"], sc.err, cen, cam.campos, cam.fy,
                             budget - ref["update"]["streamed_bytes"], pt.frame - 1)
        got = r.debug(v.DBG_PT_SLOT, np.int32).reshape(P, 1)
        np.testing.assert_array_equal(got, pt.slot)
        np.testing.assert_array_equal(r.debug(v.DBG_PT_LAST, np.int32), pt.last_used)
        np.testing.assert_array_equal(r.debug(v.DBG_PT_LOD, np.int32), pt.lod)
        pool = r.debug(v.DBG_POOL, np.uint8).reshape(P, -1)
        for (pg, l, e, s) in copies:
            np.testing.assert_array_equal(pool[e], host[pg])
    assert r.stats()["acc_prefetched_pages"] > 0


def test_prefetch_placement_parity_lod(v):
    """As above on a city scene with three LOD levels (pages of 512, fanout 8)
    and LOD on: the level of each prefetch candidate comes from the
    screen-space-error rule on the page's sphere, so levels 1 and 2 are
    prefetched too (packed eight or 64 to an entry); the page table and the
    pool's sub-slots equal the oracle's after every frame."""
    from _common import city_cam, city_scene
    raw, sc = city_scene(levels=3, fanout=8, page_size=512)
    scene = import_scene(v, raw, sc)
    # a pool larger than the view's demand and a budget that catches up with
    # it after a few frames, so budget and unused entries are left to prefetch
    n_out = 128
    W, H = 320, 180
    P = 200
    rec = scene.info.record_bytes
    budget = 60 * 512 * rec
    r = v.Renderer(scene, v.RenderConfig(max_width=W, max_height=H, lod=True, staging_bytes=budget, tau0=16.0),
                   pool_slots=P)
    p = v.Prefetcher(v.MlpShape(n_in=12 + n_out // 16, n_hidden=32, n_out=n_out, max_batch=1, seed=1, lr=0.0))
    rng = np.random.default_rng(9)
    b3 = rng.permutation(n_out).astype(np.float32) / n_out - 0.3
    Pp = p.params()
    Pp["W3"][:] = 0
    Pp["b3"][:] = b3
    p.set_params(Pp)
    rp = rs.ResidencyParams(n_entries=P, page_size=512, levels=3, fanout=8, record_bytes=rec, budget_bytes=budget,
                            lod=True, tau0=16.0)
    pt = rs.PageTable(rp)
    cen = rs.page_centroids(sc)
    cams = [city_cam(160.0, k, width=W, height=H) for k in range(8)]
    host = [scene.pages(l) for l in range(3)]
    levels_seen = set()
    for t, cam in enumerate(cams):
        prev = cams[t - 1] if t else cam
        r.render_feedback([cam])
        r.update_residency()
        v.vm3dgs_prefetch(r, p, cam, prev, 0.0)
        ref = oracle.frame(sc, pt, cam, ds=4, render_image=False)
        d2 = ((cen[:, :3] - cam.campos.astype(np.float32)) ** 2).sum(1)
        base = min(max(int(np.argmin(d2)) - n_out // 2, 0), max(sc.n_pages - n_out, 0))
        copies = rs.prefetch(pt, b3, base, 0.0, ref["req"], sc.err, cen, cam.campos, cam.fy,
                             budget - ref["update"]["streamed_bytes"], pt.frame - 1)
        levels_seen |= {l for (_, l, _, _) in copies}
        np.testing.assert_array_equal(r.debug(v.DBG_PT_SLOT, np.int32).reshape(P, 64), pt.slot)
        np.testing.assert_array_equal(r.debug(v.DBG_PT_LAST, np.int32), pt.last_used)
        np.testing.assert_array_equal(r.debug(v.DBG_PT_LOD, np.int32), pt.lod)
        pool = r.debug(v.DBG_POOL, np.uint8).reshape(P, -1)
        for (pg, l, e, s_) in copies:
            blk = host[l][pg]
            np.testing.assert_array_equal(pool[e, s_ * len(blk):(s_ + 1) * len(blk)], blk)
    assert r.stats()["acc_prefetched_pages"] > 0
    assert levels_seen & {1, 2}, levels_seen


def test_prefetcher_reduces_misses(v):
    """Trained on the renderer's own feedback over seeded flythroughs (half of
    them with abrupt 90 degree turns every 15 frames), labels = pages needed in
    the next 15 frames; evaluated on held-out turning paths with a small pool
    (150 slots of 512 Gaussians) and a 10-page copy budget per frame: fewer
    misses per frame than feedback alone, with some prefetched pages used."""
    import torch
    from paper_2506_19415_b300 import prefetch_train as ptr
    raw, sc = _blob_scene()
    scene = import_scene(v, raw, sc)
    n_out = 256
    W, H = 480, 270
    rec = scene.info.record_bytes
    cfg = v.RenderConfig(max_width=W, max_height=H, lod=False, staging_bytes=10 * 512 * rec)
    P = 150
    r = v.Renderer(scene, cfg, pool_slots=P)
    train_paths = [scenegen.random_fly_path(80, seed=100 + k, lo=0.0, hi=40.0, width=W, height_px=H, speed=0.3,
                                            turn_every=(15 if k % 2 else 0)) for k in range(40)]
    test_paths = [scenegen.random_fly_path(60, seed=900 + k, lo=0.0, hi=40.0, width=W, height_px=H, speed=0.3,
                                           turn_every=15) for k in range(6)]
    X, Y, M = ptr.make_dataset(v, r, train_paths, n_out, 12 + n_out // 16, horizon=15)
    p = v.Prefetcher(v.MlpShape(n_in=12 + n_out // 16, n_hidden=128, n_out=n_out, max_batch=128, seed=4, lr=2e-3))
    curve = ptr.train(p, X, Y, M, steps=800, batch=128)
    assert curve[-1] < 0.5 * curve[0]
    cs = torch.cuda.Stream()
    a = ptr.evaluate(v, v.Renderer(scene, cfg, pool_slots=P), test_paths, None, copy_stream=cs)
    b = ptr.evaluate(v, v.Renderer(scene, cfg, pool_slots=P), test_paths, p, threshold=-1.0, copy_stream=cs)
    print("feedback only", a, "with prefetcher", b)
    assert b["prefetched_pages_per_frame"] > 0 and b["prefetch_hits_per_frame"] > 0
    assert b["misses_per_frame"] < 0.95 * a["misses_per_frame"]
