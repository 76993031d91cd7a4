"""The BF16 predictor kernels against the FP64 oracle (oracle/mlp.py), and a
training run on pairs the integrator logs itself.

Tolerances: the kernels take BF16 operands (unit roundoff 2^-8 = 3.9e-3) with
FP32 accumulation; the oracle is given the same BF16-rounded inputs and
weights, so the remaining difference comes from rounding the two hidden
activations and the back-propagated deltas to BF16 (a few 2^-8 relative).
Gradients must agree to 3e-2 in relative norm per tensor with cosine > 0.999
for batches of hundreds of samples or more; with a handful of samples the
weight-gradient sums cancel and the BF16 rounding shows through amplified, so
batches under 256 get 0.15 and cosine > 0.99.  The loss must agree to 1e-2
relative; predicted classes wherever the oracle's top two logits differ by more
than 0.1.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2102_10983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2102_10983_gb300 import native  # noqa: E402


def _bf16(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    phi = np.stack([np.arcsinh(np.abs(rng.normal(0, 50, n))), np.arcsinh(np.abs(rng.normal(0, 50, n))),
                    np.arcsinh(rng.normal(0, 30, n)), np.arcsinh(rng.normal(0, 30, n)),
                    np.arcsinh(rng.normal(0, 0.2, n)), np.log(1 + np.abs(rng.normal(0, 30, n)))], 1)
    y = rng.integers(0, 8, n).astype(np.uint8)
    return phi.astype(np.float32), y


@pytest.mark.parametrize("n", [3001, 16, 1])
def test_gradients_match_oracle(n):
    P = omlp.init_params(5)
    for k in P:
        if k.startswith("b"):
            P[k] = np.random.default_rng(2).normal(0, 0.1, P[k].shape)
    phi, y = _batch(n, 4)
    net = native.Predictor()
    net.set_params(native.pack_params(P))
    g, loss = net.grad(torch.as_tensor(phi, device="cuda"), torch.as_tensor(y, device="cuda"))
    Pb = {k: (_bf16(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
          for k, v in P.items()}
    lref, gref = omlp.loss_and_grads(Pb, _bf16(phi), y)
    gg = native.unpack_params(g)
    tol, cos = (3e-2, 0.999) if n >= 256 else (0.15, 0.99)
    assert abs(loss - lref) <= 1e-2 * abs(lref), (loss, lref)
    for k in gref:
        a, b = gg[k].reshape(-1), gref[k].reshape(-1)
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.linalg.norm(a) < 1e-6
            continue
        assert np.linalg.norm(a - b) <= tol * nb, (k, np.linalg.norm(a - b) / nb)
        assert a @ b / (np.linalg.norm(a) * nb) > cos, k
    net.close()


def test_inference_matches_oracle():
    P = omlp.init_params(9)
    phi, _ = _batch(5000, 8)
    net = native.Predictor()
    net.set_params(native.pack_params(P))
    pred = torch.empty(len(phi), dtype=torch.uint8, device="cuda")
    net.infer(torch.as_tensor(phi, device="cuda"), pred)
    Pb = {k: (_bf16(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
          for k, v in P.items()}
    z, _ = omlp.forward(Pb, _bf16(phi))
    zs = np.sort(z, axis=1)
    clear = (zs[:, -1] - zs[:, -2]) > 0.1
    got = pred.cpu().numpy()
    assert clear.mean() > 0.8
    np.testing.assert_array_equal(got[clear], np.argmax(z, axis=1)[clear])
    net.close()


def test_features_kernel_matches_definition():
    """pic_features against the stated transform, with E and B extrapolated to
    t_{n+1} (theta = 3/2) by the oracle's own weights and a tent gather."""
    import oracle
    wl = W.Workload(name="feat", n_particles=2000, a0=100.0, dt=W.DT75, dx=W.DT75 / 0.99,
                    psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=2 * math.pi, seed=3)
    p = wl.order
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=native.PIC_MIXED,
                              capacity=wl.n_particles, window=wl.window, ring_levels=p + 2)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    E, B, i0 = wl.levels(-p, 60 + p)
    for r in range(p):
        integ.pic_fields_upload(r - p, i0[r], E[r], B[r])
    for s in range(60):
        integ.pic_fields_upload(s, i0[s + p], E[s + p], B[s + p])
        integ.pic_push_step(s, 1, want_stats=False)
    phi = torch.empty((wl.n_particles, 6), dtype=torch.float32, device="cuda")
    native.features(integ, 59, phi)
    x, px, py, pz, st = integ.read_numpy()
    integ.close()
    wE, wB = oracle.lagrange(p, "E", 1.5), oracle.lagrange(p, "B", 1.5)
    # rows 59..62 of E/B hold levels 56..59, each on its own window origin
    s_ = x / wl.dx

    def gather(F, w, s):
        j = np.floor(s).astype(np.int64)
        f = s - j
        v0 = sum(w[l] * F[59 + l][j - i0[59 + l]] for l in range(p + 1))
        v1 = sum(w[l] * F[59 + l][j + 1 - i0[59 + l]] for l in range(p + 1))
        return v0 + f * (v1 - v0)

    want = omlp.features(gather(E, wE, s_), gather(B, wB, s_ - 0.5), px, py, pz)
    got = phi.cpu().numpy().astype(np.float64)
    alive = (st & native.PIC_STATUS_LOST) == 0
    assert alive.mean() > 0.9
    np.testing.assert_allclose(got[alive], want[alive], rtol=2e-5, atol=2e-4)


@pytest.mark.parametrize("n", [4000, 37])
def test_fused_prediction_equals_features_then_inference(n):
    """pic_predict (features and inference in one kernel) gives exactly the
    classes of pic_features followed by pic_mlp_infer, including ragged tails
    of the 32-particle warp tiles, with a network trained a little so its
    weights are not the initial ones."""
    wl = W.Workload(name="fused", n_particles=n, a0=150.0, dt=W.DT75, dx=W.DT75 / 0.99,
                    psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=2 * math.pi,
                    thermal_sigma=W.MAXWELL_10KEV_SIGMA, seed=5)
    p = wl.order
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=native.PIC_MIXED,
                              capacity=wl.n_particles, window=wl.window, ring_levels=p + 2)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    E, B, i0 = wl.levels(-p, 40 + p)
    for r in range(p):
        integ.pic_fields_upload(r - p, i0[r], E[r], B[r])
    for s in range(40):
        integ.pic_fields_upload(s, i0[s + p], E[s + p], B[s + p])
        integ.pic_push_step(s, 1, want_stats=False)
    net = native.Predictor(seed=3)
    phi_t, y_t = _batch(4096, 9)
    for _ in range(20):
        net.train_step(torch.as_tensor(phi_t, device="cuda"), torch.as_tensor(y_t, device="cuda"), 3e-3)
    phi = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    native.features(integ, 39, phi)
    want = torch.empty(n, dtype=torch.uint8, device="cuda")
    net.infer(phi, want)
    got = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    native.predict(integ, net, 39, got)
    torch.cuda.synchronize()
    integ.close()
    net.close()
    assert torch.equal(got, want)


def test_training_on_logged_pairs_learns_the_next_k():
    """Log (features after step n, k of step n+1) from a run of the integrator,
    train on the GPU, and predict held-out pairs: the network must beat the
    'same k as last step' rule on the steps where k changes."""
    wl = W.Workload(name="log", n_particles=65536, a0=100.0, dt=W.DT75, dx=W.DT75 / 0.99,
                    psi_max=0.01, order=3, n_steps=0, x_lo=0.0, x_hi=4 * math.pi, seed=6,
                    window=512, lead=120)
    p = wl.order
    integ = native.Integrator(wl.dt, wl.dx, wl.psi_max, order=p, precision=native.PIC_MIXED,
                              schedule=native.PIC_SCHED_BINNED, capacity=wl.n_particles,
                              window=wl.window, ring_levels=p + 3)
    ini = wl.particles()
    integ.pic_particles_write(ini.x, ini.px, ini.py, ini.pz)
    steps = 400
    E, B, i0 = wl.levels(-p, steps + p)
    for r in range(p):
        integ.pic_fields_upload(r - p, i0[r], E[r], B[r])
    feats, labels, prev = [], [], []
    phi = torch.empty((wl.n_particles, 6), dtype=torch.float32, device="cuda")
    st = torch.empty(wl.n_particles, dtype=torch.uint8, device="cuda")
    for s in range(steps):
        integ.pic_fields_upload(s, i0[s + p], E[s + p], B[s + p])
        integ.pic_push_step(s, 1, want_stats=False)
        integ.pic_particles_read(status=st)
        k_now = (st & 0x7F).clone()
        if s > 0:
            labels.append(k_now)           # k of step s for the features after step s-1
            prev.append(k_prev)
        if s < steps - 1:
            native.features(integ, s, phi)
            feats.append(phi.clone())
        k_prev = k_now
    integ.close()
    X = torch.cat(feats[: len(labels)])
    Y = torch.cat(labels).to(torch.uint8)
    K0 = torch.cat(prev)
    alive = torch.isfinite(X).all(1)
    X, Y, K0 = X[alive], Y[alive], K0[alive]
    # keep every pair whose k is nonzero or changed, and a sample of the rest
    interesting = (Y > 0) | (K0 > 0)
    g = torch.Generator(device="cuda").manual_seed(0)
    keep = interesting | (torch.rand(len(Y), device="cuda", generator=g) < 0.02)
    X, Y, K0 = X[keep], Y[keep], K0[keep]
    perm = torch.randperm(len(Y), device="cuda", generator=g)
    X, Y, K0 = X[perm], Y[perm], K0[perm]
    n_tr = int(0.8 * len(Y))
    net = native.Predictor(seed=1)
    losses = []
    bs = 8192
    for it in range(600):
        a = (it * bs) % max(n_tr - bs, 1)
        losses.append(net.train_step(X[a:a + bs].contiguous(), Y[a:a + bs].contiguous(), 2e-3))
    pred = torch.empty(len(Y) - n_tr, dtype=torch.uint8, device="cuda")
    net.infer(X[n_tr:].contiguous(), pred)
    yt, k0t = Y[n_tr:], K0[n_tr:]
    acc_net = (pred == yt).float().mean().item()
    acc_prev = (k0t == yt).float().mean().item()
    changed = k0t != yt
    acc_net_changed = (pred[changed] == yt[changed]).float().mean().item()
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    assert acc_net > 0.85, acc_net
    assert acc_net_changed > 0.5, (acc_net_changed, changed.float().mean().item(), acc_prev)
    net.close()
