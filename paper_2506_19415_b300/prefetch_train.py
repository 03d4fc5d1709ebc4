"""Training and evaluation of the learned page prefetcher.

Orchestration only: every computation runs in the library's kernels
(vm3dgs_render_feedback, vm3dgs_prefetch_features / _labels, the
prefetcher's forward and training step, vm3dgs_update_residency,
vm3dgs_prefetch); torch tensors hold the dataset on the device.

Dataset (from the renderer's own visibility feedback): for every frame t of
a flythrough, x_t = network input of frame t (camera motion + histogram of the
pages requested at t over the page window around the camera) and
y_t = pages of that window requested in any of the frames t+1 .. t+horizon.
"""
from __future__ import annotations

import time

import numpy as np


def make_dataset(v, r, paths, n_out, n_in, horizon=1):
    """Feedback-only passes over the paths; returns device tensors X, Y, M."""
    import torch
    dev = r.pool.device
    n = sum(len(p) - 1 for p in paths)
    X = torch.empty((n, n_in), dtype=torch.float32, device=dev)
    Y = torch.zeros((n, n_out), dtype=torch.float32, device=dev)
    M = torch.empty((n, n_out), dtype=torch.float32, device=dev)
    T = max(len(p) for p in paths)
    base = torch.empty((T, 1), dtype=torch.int32, device=dev)
    k0 = 0
    for path in paths:
        for t, cam in enumerate(path):
            r.render_feedback([cam])
            # frame t is within the horizon of the samples of frames t-horizon .. t-1:
            # the labels kernel ORs this frame's requests into theirs
            for s_ in range(max(0, t - horizon), t):
                k = k0 + s_
                v.vm3dgs_prefetch_labels(r, n_out, base[s_], Y[k], M[k], accumulate=True)
            if t + 1 < len(path):
                v.vm3dgs_prefetch_features(r, n_out, cam, path[t - 1] if t > 0 else cam, X[k0 + t], base[t])
        k0 += len(path) - 1
    torch.cuda.synchronize()
    return X, Y, M


def train(p, X, Y, M, steps=1000, batch=256, seed=0):
    """Adam on random minibatches; returns the loss curve (every 50 steps)."""
    import torch
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    n = X.shape[0]
    batch = min(batch, p.shape.max_batch, n)
    p._fixed_mask_sum = float(M[:1].sum().item()) * batch
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    curve = []
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), device=X.device, generator=g)
        p.train_step(X[idx], Y[idx], M[idx], loss_out=loss)
        if s % 50 == 0 or s == steps - 1:
            curve.append(float(loss.item()))
    del p._fixed_mask_sum
    return curve


def evaluate(v, r, paths, p=None, threshold=0.0, copy_stream=None):
    """Runs the virtual-memory frames over the paths (feedback -> residency,
    no image) with or without prefetching; returns misses/frame and the
    mean per-frame time of the copies the frame waits for."""
    import torch
    r.timing(True)
    r.timing_read()
    r.reset_sums()
    frames = 0
    for path in paths:
        for t, cam in enumerate(path):
            r.render_feedback([cam])
            r.update_residency(None, copy_stream)
            if p is not None:
                v.vm3dgs_prefetch(r, p, cam, path[t - 1] if t > 0 else cam, threshold, None, copy_stream)
            frames += 1
    torch.cuda.synchronize()
    ms, _ = r.timing_read()
    r.timing(False)
    st = r.stats()
    return dict(frames=frames, misses_per_frame=st["acc_missing"] / max(frames, 1),
                stall_ms_per_frame=ms[v.STAGES.index("stream")] / max(frames, 1),
                prefetched_pages_per_frame=st["acc_prefetched_pages"] / max(frames, 1),
                prefetch_hits_per_frame=st["acc_prefetch_hits"] / max(frames, 1),
                requested_per_frame=st["acc_requested"] / max(frames, 1))
