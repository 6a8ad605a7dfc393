"""Batched RK3-substep solves (fork/join and one CUDA graph) and the autotuner."""
import json
import math
import os
import time

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import batch as B
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu


def _inputs(plans, seed0):
    return [torch.from_numpy(S.gaussian(seed0 + i, p.shape)).cuda() for i, p in enumerate(plans)]


def _oracle_grid(plan, beta=1.8):
    """The oracle's own grid for a plan: spacings derived by the oracle from
    the same synthetic faces (cell-centred, or node-centred for DF walls)."""
    if plan.bc[4] == O.BC_DF:
        dzc, dzf = O.face_spacings(S.tanh_faces(plan.nz + 1, beta))
    else:
        dzc, dzf = O.cell_spacings(S.tanh_faces(plan.nz, beta))
    return O.Grid(plan.nx, plan.ny, plan.nz, plan.dx, plan.dy, dzc, dzf, plan.bc)


def test_batch_matches_single_solves_and_oracle(cuda_device):
    domains = [(32, 16, 16), (48, 32, 24), (64, 32, 40)]
    alphas = [1e-4, 1e-3, 1e-4]
    batch, plans, tags = B.rk3_substep_batch(domains, alphas)
    fs = _inputs(plans, 4000)
    us = [torch.empty_like(f) for f in fs]
    batch.solve(fs, us)
    torch.cuda.synchronize()
    us2 = [torch.empty_like(f) for f in fs]
    batch.solve(fs, us2)
    torch.cuda.synchronize()
    assert batch.grouped()                 # FP32 + refinement plans: grouped stage launches
    report = []
    for (d, name), plan, f, u, u2 in zip(tags, plans, fs, us, us2):
        ref = plan.poisson(f) if name == "p" else plan.helmholtz(alphas[d], f)
        torch.cuda.synchronize()
        rel = float(torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref))
        rel2 = float(torch.linalg.vector_norm(u - u2) / torch.linalg.vector_norm(ref))
        report.append((d, name, rel, rel2))
    print("batch vs single:", report)
    for (d, name), plan, f, u in zip(tags, plans, fs, us):
        g = _oracle_grid(plan)
        o = O.solve(f.cpu().numpy(), g, None if name == "p" else alphas[d])
        assert O.rel_l2(u.cpu().numpy(), o) <= 1e-10, (d, name)
    # bitwise except singular Poisson solves, whose refinement gauge sum is an
    # FP64 atomic reduction (order-dependent rounding, ~1e-16)
    assert all((r[2] == 0.0 and r[3] == 0.0) if r[1] != "p" else (r[2] <= 1e-13 and r[3] <= 1e-13) for r in report), report


def test_batch_graph_replay(cuda_device):
    domains = [(32, 16, 16), (64, 32, 40)]
    batch, plans, tags = B.rk3_substep_batch(domains, [1e-3, 1e-4])
    fs = _inputs(plans, 4100)
    direct = [torch.empty_like(f) for f in fs]
    batch.solve(fs, direct)
    us = [torch.full_like(f, float("nan")) for f in fs]
    st = batch.capture(fs, us)
    assert batch.grouped() and batch.graph_nodes() <= 60     # one launch per stage and kernel variant
    for _ in range(2):
        batch.launch(st)
        st.synchronize()
        for (d, name), a, b in zip(tags, us, direct):
            if name == "p":
                assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) <= 1e-13
            else:
                assert torch.equal(a, b)


@pytest.mark.parametrize("autotune", [True, False])
def test_grouped_and_fork_join_batches_agree(cuda_device, autotune):
    """The grouped stage launches against the fork/join of per-solve launches
    over streams: the same kernels' arithmetic per solve, so bit for bit
    except singular Poisson solves (order of the FP64 gauge-sum atomics).
    With the default schedules the w solve of the third domain (32 wall-node
    rows, two full z segments of 16) runs the full-segment z kernel alone and
    the ragged-segment kernel in the grouped launch."""
    domains = [(48, 32, 24), (96, 64, 40), (64, 48, 33)]
    alphas = [1e-4, 1e-3, 1e-4]
    batch, plans, tags = B.rk3_substep_batch(domains, alphas, autotune=autotune)
    fs = _inputs(plans, 4200)
    ug = [torch.empty_like(f) for f in fs]
    batch.solve(fs, ug)
    assert batch.grouped()
    batch.set_grouped(False)
    uf = [torch.empty_like(f) for f in fs]
    batch.solve(fs, uf)
    torch.cuda.synchronize()
    assert not batch.grouped()
    st = batch.capture(fs, [torch.empty_like(f) for f in fs])
    nodes_fork = batch.graph_nodes()
    batch.set_grouped(True)
    batch.capture(fs, [torch.empty_like(f) for f in fs], st)
    nodes_grouped = batch.graph_nodes()
    print(f"graph nodes: fork/join {nodes_fork}, grouped {nodes_grouped}")
    assert nodes_grouped <= 60 < nodes_fork
    for (d, name), a, b in zip(tags, ug, uf):
        if name == "p":
            assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) <= 1e-13, (d, name)
        else:
            assert torch.equal(a, b), (d, name)


def test_autotune_sets_and_caches_a_schedule(cuda_device, tmp_path):
    plan = cs.channel_plan(192, 96, 128, beta=1.8)
    plan.set_precision(cs.FP32)
    cache = tmp_path / "tune.json"
    sched = plan.autotune(str(cache))
    assert cache.exists() and len(json.loads(cache.read_text())) == 1
    assert all(v >= 0 for v in sched)
    plan2 = cs.channel_plan(192, 96, 128, beta=1.8)
    plan2.set_precision(cs.FP32)
    assert plan2.autotune(str(cache)) == sched              # served from the cache
    f = torch.from_numpy(S.gaussian(77, plan.shape)).cuda()
    g = _oracle_grid(plan)
    assert O.rel_l2(plan.poisson(f.float()).double().cpu().numpy(), O.solve(f.cpu().numpy(), g)) <= 1e-5


def test_rk3_substep_16_domains_graph(cuda_device):
    """The 16 uneven channel domains (64^3 ... 384x192x160): u, v, w Helmholtz
    (alpha 1e-4 / 1e-3 alternating) and p Poisson per domain, FP32 + refinement,
    one CUDA graph; every one of the 64 solves checked against the oracle."""
    alphas = [1e-4 if d % 2 == 0 else 1e-3 for d in range(len(S.BATCH_DOMAINS))]
    batch, plans, tags = B.rk3_substep_batch(S.BATCH_DOMAINS, alphas)
    fs = [torch.from_numpy(S.gaussian(4000 + 10 * d + i, p.shape)).cuda()
          for (d, _), i, p in zip(tags, range(len(plans)), plans)]
    us = [torch.empty_like(f) for f in fs]
    st = batch.capture(fs, us)
    assert batch.grouped() and batch.graph_nodes() <= 60
    batch.launch(st)
    st.synchronize()
    worst = {}
    for k, (d, name) in enumerate(tags):
        o = O.solve(fs[k].cpu().numpy(), _oracle_grid(plans[k]), None if name == "p" else alphas[d])
        rel = O.rel_l2(us[k].cpu().numpy(), o)
        worst[name] = max(worst.get(name, 0.0), rel)
        assert rel <= 1e-10, (d, name, rel)
    print("worst rel err per field over the 16 domains:", worst)
    for _ in range(2):
        batch.launch(st)
    st.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        batch.launch(st)
    st.synchronize()
    dt = (time.perf_counter() - t0) / reps
    pts = sum(p.numel for p in plans)
    print(f"RK3 substep, 16 domains, {len(plans)} solves, {batch.graph_nodes()} graph nodes: "
          f"{dt * 1e3:.2f} ms, {pts / dt / 1e9:.2f} Gpoint-solves/s")


def test_fast_refinement_batch_takes_the_fork_join(cuda_device):
    """Plans in the fast refinement mode are batched by the fork/join over
    streams (the grouped stages are built for the exact-residual mode); the
    results stay within the refinement tolerance of the oracle."""
    domains = [(48, 32, 24), (64, 32, 40)]
    batch, plans, tags = B.rk3_substep_batch(domains, [1e-3, 1e-4], precision=cs.FP32_REFINE_FAST, autotune=False)
    fs = _inputs(plans, 4300)
    us = [torch.empty_like(f) for f in fs]
    batch.solve(fs, us)
    torch.cuda.synchronize()
    assert not batch.grouped()
    for (d, name), plan, f, u in zip(tags, plans, fs, us):
        o = O.solve(f.cpu().numpy(), _oracle_grid(plan), None if name == "p" else [1e-3, 1e-4][d])
        assert O.rel_l2(u.cpu().numpy(), o) <= 1e-10, (d, name)
