"""GPU parity of the projection operators, the differentiable solve and the
learned closure against the FP64 CPU oracle."""
import math
import time

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import autograd as AG
from paper_2411_09364_gb300 import closure as CL
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu


def channel_pair(nx, ny, nz, beta=1.8, precision=cs.FP64):
    zf = S.tanh_faces(nz, beta)
    odzc, odzf = O.cell_spacings(zf)
    gdzc, gdzf = cs.cell_spacings(zf)
    bc = (0, 0, 0, 0, 1, 1)
    g = O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, odzc, odzf, bc)
    plan = cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, gdzc, gdzf, precision)
    return g, plan


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def host(t):
    return t.double().cpu().numpy()


def maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_div_grad_and_transposes(cuda_device):
    g, plan = channel_pair(24, 16, 12)
    u, v, w = S.velocity_field(7, 24, 16, 12)
    d = AG.divergence(plan, dev(u), dev(v), dev(w))
    assert maxrel(host(d), O.divergence(u, v, w, g)) < 1e-12
    phi = S.gaussian(8, (12, 16, 24))
    gx, gy, gz = AG.gradient(plan, dev(phi))
    ox, oy, oz = O.gradient(phi, g)
    assert max(maxrel(host(gx), ox), maxrel(host(gy), oy), maxrel(host(gz), oz)) < 1e-12
    sx, sy, sz = AG.gradient(plan, dev(phi), sub=(dev(u), dev(v), dev(w)))
    assert maxrel(host(sz), w - oz) < 1e-12 and maxrel(host(sx), u - ox) < 1e-12
    tu, tv, tw = AG.divergence_T(plan, dev(phi))
    ou, ov, ow = O.divergence_T(phi, g)
    assert max(maxrel(host(tu), ou), maxrel(host(tv), ov), maxrel(host(tw), ow)) < 1e-12
    gt = AG.gradient_T(plan, dev(u), dev(v), dev(w))
    assert maxrel(host(gt), O.gradient_T(u, v, w, g)) < 1e-12


@pytest.mark.parametrize("precision,tol", [(cs.FP64, 1e-12), (cs.FP32, 1e-5)])
def test_projection_matches_oracle(cuda_device, precision, tol):
    g, plan = channel_pair(32, 16, 24, precision=precision)
    dt = torch.float64 if precision == cs.FP64 else torch.float32
    vel = list(S.velocity_field(9, 32, 16, 24))
    out = AG.project_forward(plan, *[dev(a, dt) for a in vel])
    ref = O.project_velocity(vel, g)
    err = math.sqrt(sum(((host(o) - r) ** 2).sum() for o, r in zip(out, ref)) / sum((r ** 2).sum() for r in ref))
    assert err < tol
    div = AG.divergence(plan, *[o for o in out])
    assert float(div.abs().max()) < (1e-9 if precision == cs.FP64 else 1e-2) * float(
        AG.divergence(plan, *[dev(a, dt) for a in vel]).abs().max())


def test_config2_rhs_from_gpu_divergence(cuda_device):
    """512 x 256 x 192 channel: the RHS is the divergence of a Gaussian
    staggered velocity, computed by each side with its own operator."""
    nx, ny, nz = 512, 256, 192
    g, plan = channel_pair(nx, ny, nz, beta=1.8)
    u, v, w = S.velocity_field(2000, nx, ny, nz)
    ref = O.solve(O.divergence(u, v, w, g), g)
    dg = AG.divergence(plan, dev(u), dev(v), dev(w))
    p = host(plan.poisson(dg))
    assert O.rel_l2(p, ref) <= 1e-12
    plan.set_precision(cs.FP32_REFINE, 2)
    assert O.rel_l2(host(plan.poisson(dg)), ref) <= 1e-10


def test_config5_differentiable_projection(cuda_device):
    """256 x 128 x 128 stretched channel, FP32: loss = sum(w * p) with p = S f;
    the autograd backward (adjoint kernel) against the oracle's transposed
    solve and central finite differences (eps = 1e-3, 32 seeded entries,
    evaluated with the FP64 solve)."""
    nx, ny, nz = 256, 128, 128
    g, plan32 = channel_pair(nx, ny, nz, beta=1.8, precision=cs.FP32)
    _, plan64 = channel_pair(nx, ny, nz, beta=1.8, precision=cs.FP64)
    f_np = S.gaussian(5000, (nz, ny, nx))
    w_np = S.gaussian(5001, (nz, ny, nx))
    f = dev(f_np, torch.float32).requires_grad_(True)
    w = dev(w_np, torch.float32)
    p = AG.poisson_solve(f, plan32)
    (w * p).sum().backward()
    grad = host(f.grad)
    ref = O.solve_T(w_np, g)
    assert O.rel_l2(grad, ref) <= 1e-5
    # central differences with the FP64 solve
    rng = np.random.default_rng(5002)
    idx = rng.choice(f_np.size, 32, replace=False)
    f64 = dev(f_np)
    w64 = dev(w_np)
    eps = 1e-3
    flat = f64.view(-1)
    fd = []
    for i in idx:
        old = float(flat[i])
        flat[i] = old + eps
        lp = float(torch.dot(w64.view(-1), plan64.poisson(f64).view(-1)))
        flat[i] = old - eps
        lm = float(torch.dot(w64.view(-1), plan64.poisson(f64).view(-1)))
        flat[i] = old
        fd.append((lp - lm) / (2 * eps))
    fd = np.array(fd)
    assert np.abs(grad.reshape(-1)[idx] - fd).max() <= 1e-4 * np.abs(grad).max()
    assert np.abs(ref.reshape(-1)[idx] - fd).max() <= 1e-6 * np.abs(ref).max()
    # throughput of forward + backward (FP32)
    for _ in range(3):
        f.grad = None
        (w * AG.poisson_solve(f, plan32)).sum().backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 10
    for _ in range(reps):
        f.grad = None
        (w * AG.poisson_solve(f, plan32)).sum().backward()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    print(f"config5 forward+backward: {dt * 1e3:.3f} ms, {nx * ny * nz / dt / 1e9:.2f} Gpoints/s")


def _closure_setup(nx, ny, nz, seed):
    g, plan = channel_pair(nx, ny, nz, beta=1.5, precision=cs.FP32)
    vel_np = list(S.velocity_field(seed, nx, ny, nz))
    vel = [dev(a, torch.float32) for a in vel_np]
    return g, plan, vel_np, vel


def test_closure_loss_and_gradient_match_oracle(cuda_device):
    g, plan, vel_np, vel = _closure_setup(32, 16, 16, 300)
    net = CL.StencilClosure(plan)
    theta_np = 0.02 * np.random.default_rng(301).standard_normal((3, 27))
    net.theta.copy_(torch.from_numpy(theta_np).float())
    target_np = O.project_velocity(O.hidden_operator(vel_np), g)
    target = net.target(vel)
    terr = math.sqrt(sum(((host(t) - r) ** 2).sum() for t, r in zip(target, target_np))
                     / sum((r ** 2).sum() for r in target_np))
    assert terr < 1e-5
    loss = net.loss(vel, target, with_grad=True)
    ref_loss, ref_grad = O.closure_loss_grad(theta_np.astype(np.float32).astype(np.float64), vel_np, target_np, g)
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    grad = net.gacc.cpu().numpy()
    assert np.linalg.norm(grad - ref_grad) <= 1e-3 * np.linalg.norm(ref_grad)


def test_closure_training_gains_over_the_method_without_it(cuda_device):
    nx, ny, nz = 64, 32, 32
    g, plan, _, _ = _closure_setup(nx, ny, nz, 0)
    net = CL.StencilClosure(plan, lr=2e-2)
    train = []
    for s in range(4):
        vel = [dev(a, torch.float32) for a in S.velocity_field(400 + s, nx, ny, nz)]
        train.append((vel, net.target(vel)))
    held = []
    for s in range(2):
        vel = [dev(a, torch.float32) for a in S.velocity_field(500 + s, nx, ny, nz)]
        held.append((vel, net.target(vel)))
    zero = torch.zeros((3, 27), device="cuda")
    base = np.mean([net.loss(v, t, theta=zero) for v, t in held])
    losses = [net.step(*train[i % 4]) for i in range(200)]
    trained = np.mean([net.loss(v, t) for v, t in held])
    print(f"closure held-out loss: without {base:.4e}, trained {trained:.4e} (ratio {trained / base:.3f}); "
          f"train loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert trained < 0.3 * base
    assert losses[-1] < 0.3 * losses[0]
