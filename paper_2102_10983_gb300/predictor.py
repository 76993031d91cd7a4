"""Training data and training loop of the learned sub-cycle-count predictor.

The integrator logs its own (features, next-step k) pairs: after macro step n,
pic_features gives each electron's (|E|, |B|, p, gamma) features from the
levels it has, and the criterion of step n+1 (read back from the status bytes)
gives the label.  Training runs the hand-written BF16 kernels through
pic_mlp_train_step.  Everything here is device tensors and C-ABI calls.
"""
from __future__ import annotations

import numpy as np

from . import native
from .workloads import Workload


def log_pairs(wl: Workload, steps: int, keep_quiet: float = 0.02, seed: int = 0):
    """Run `wl` for `steps` macro steps (mixed form, binned schedule) and return
    (phi [N, 6] float32, k_next [N] uint8, k_prev [N] uint8) on the device.

    All pairs with k_next > 0 or k_prev > 0 are kept; of the quiet rest (both 0)
    a fraction `keep_quiet` is kept.
    """
    import torch
    p = wl.order
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=native.PIC_MIXED,
                              schedule=native.PIC_SCHED_BINNED, capacity=wl.n_particles,
                              window=wl.window, ring_levels=p + 3)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    E, B, i0 = wl.levels(-p, steps + p)
    for r in range(p):
        integ.pic_fields_upload(r - p, i0[r], E[r], B[r])
    n = wl.n_particles
    phi = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(seed)
    xs, ys, ks = [], [], []
    feats_prev = None
    k_prev = None
    for s in range(steps):
        integ.pic_fields_upload(s, i0[s + p], E[s + p], B[s + p])
        integ.pic_push_step(s, 1, want_stats=False)
        integ.pic_particles_read(status=st)
        k_now = (st & 0x7F).clone()
        alive = (st & native.PIC_STATUS_LOST) == 0
        if feats_prev is not None:
            sel = alive & ((k_now > 0) | (k_prev > 0) |
                           (torch.rand(n, device="cuda", generator=g) < keep_quiet))
            xs.append(feats_prev[sel])
            ys.append(k_now[sel])
            ks.append(k_prev[sel])
        native.features(integ, s, phi)
        feats_prev = phi.clone()
        k_prev = k_now
    integ.close()
    return torch.cat(xs), torch.cat(ys).to(torch.uint8), torch.cat(ks).to(torch.uint8)


def train(net: "native.Predictor", X, Y, iters: int = 600, lr: float = 2e-3, batch: int = 8192,
          seed: int = 0):
    """Adam on shuffled mini-batches; returns the list of batch losses."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    perm = torch.randperm(len(Y), device="cuda", generator=g)
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    losses = []
    n = len(Y)
    for it in range(iters):
        a = (it * batch) % max(n - batch, 1)
        losses.append(net.train_step(X[a:a + batch].contiguous(), Y[a:a + batch].contiguous(), lr))
    return losses


def c1_style_training_set(n_electrons: int = 65536, steps: int = 400, seed: int = 6,
                          keep_quiet: float = 1.0):
    """Pairs from at-rest electrons in a switched-on a0 = 100 wave at dt = lambda/75
    (the test-particle configuration, in a smaller ensemble).  By default every
    pair is kept, so the classes come with their natural frequencies and the
    network's argmax only leaves k = 0 when it is confident: the schedule bins
    a particle on that prediction, and a false alarm costs work."""
    import math
    from .workloads import DT75
    wl = Workload(name="predictor_training", n_particles=n_electrons, a0=100.0, dt=DT75,
                  dx=DT75 / 0.99, psi_max=0.01, order=3, n_steps=steps, x_lo=0.0,
                  x_hi=4 * math.pi, seed=seed, window=512, lead=120)
    return log_pairs(wl, steps, keep_quiet=keep_quiet)
