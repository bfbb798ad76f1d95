"""GPU tests of the refined solve's device-side schedule, of the FISTA
checkpoint and of the TV prox's bounded grid barrier, through the C-ABI.

The refined solve (BF16 increments of the gradient with exact two-term BF16
resyncs) is held to the FP32 solve's bound against the FP64 oracle: FISTA
iterates after the tiny workload's 20 iterations within 1e-4 (relative L2),
with the schedule the benchmark runs (``REFINED_DEFAULTS``).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_23739_gb300 as sw
import synth

pytestmark = pytest.mark.gpu

TINY = synth.workload("tiny_16x16x24_T64_k7_N8_P2")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def tiny():
    g, s = TINY.geom, TINY.sw
    K = synth.transducer_kernel(g, seed=0)
    c_true = synth.tube_phantom(g, TINY.tubes, seed=0, per_species=True)
    clean = oracle.forward(g, s, K, c_true)
    y = clean + synth.noise_sigma(clean, TINY.snr_db) * synth.gaussian(g.y_shape(), 100)
    L = oracle.power(g, s, K, synth.gaussian(g.c_shape(), 1), 100)
    ref = oracle.fista(g, s, K, y, 1.0 / L, TINY.iters, TINY.lam_l1, TINY.lam_tv, TINY.inner)
    return g, s, K, y, 1.0 / L, ref


def _params(alpha, iters, **kw):
    return sw.SolveParams(step=alpha, lambda_l1=TINY.lam_l1, lambda_tv=TINY.lam_tv,
                          inner_iters=TINY.inner, max_iters=iters, **kw)


def test_refined_default_schedule_matches_oracle(tiny):
    """The benchmark's schedule (BF16 increments, exact gradient every 25
    iterations or when the accumulated relative step exceeds the budget):
    the tiny workload's 20 iterations within the FP32 bound of the oracle,
    with some iterations taken on BF16 increments."""
    g, s, K, y, alpha, ref = tiny
    op = sw.Operator(g, K, s, precision="bf16")
    got, stats = op.solve(dev(y), _params(alpha, TINY.iters, **sw.REFINED_DEFAULTS))
    its, resyncs = op.refine_stats()
    op.check_device()
    op.close()
    assert stats["iters"] == TINY.iters and its == TINY.iters
    assert 1 < resyncs < TINY.iters + 1  # the initial gradient, some resyncs, some increments
    assert rel(host(got), ref) <= 1e-4


def test_refined_budget_graph_equals_direct_launches(tiny):
    """Both branches of the device-side decision are captured in one graph:
    replaying it gives the iterates of launching the kernels one by one."""
    g, s, K, y, alpha, _ = tiny
    params = _params(alpha, 14, **sw.REFINED_DEFAULTS)
    op = sw.Operator(g, K, s, precision="bf16")
    op.fista_init(dev(y), params)
    op.fista_step(14)
    a = op.fista_get().clone()
    ra = op.refine_stats()
    op.use_graphs(False)
    op.fista_init(dev(y), params)
    op.fista_step(14)
    b = op.fista_get()
    assert torch.equal(a, b) and op.refine_stats() == ra
    op.close()


def test_refined_budget_profile_counts_the_branch_taken(tiny):
    """Profiled launches behind the gate count only where the device chose
    their branch: increments plus exact gradients equal the iterations."""
    g, s, K, y, alpha, _ = tiny
    op = sw.Operator(g, K, s, precision="bf16")
    op.fista_init(dev(y), _params(alpha, 30, **sw.REFINED_DEFAULTS))
    op.profile(True)
    for k in range(4):
        op.profile_read(k)
    op.fista_step(12)
    inc = op.profile_read(0)["launches"]
    exact = op.profile_read(2)["launches"]
    its, resyncs = op.refine_stats()
    op.profile(False)
    op.close()
    assert its == 12
    assert inc + exact == 12
    assert exact == resyncs - 1  # the initial exact gradient runs before the steps


@pytest.mark.parametrize("prec,kw", [("fp32", {}),
                                     ("bf16", sw.REFINED_DEFAULTS),
                                     ("bf16", {"refine_every": 4, "refine_precision": "bf16x3"})])
def test_checkpoint_resume_is_bitwise(tiny, prec, kw):
    """10 iterations, save, a fresh start of the solve, restore, 10
    iterations: the iterate of 20 straight iterations, bit for bit.  The
    restore goes into the handle that saved (the tensor-core tiling, chosen
    by timing per handle, fixes the FP32 summation order); a new FP32 handle
    (CUDA-core arithmetic, no tuning) resumes bit for bit too."""
    g, s, K, y, alpha, _ = tiny
    params = _params(alpha, 20, **kw)
    yd = dev(y)
    a = sw.Operator(g, K, s, precision=prec)
    a.fista_init(yd, params)
    a.fista_step(20)
    straight = a.fista_get().clone()
    a.fista_init(yd, params)
    a.fista_step(10)
    state = a.fista_save()
    a.fista_init(yd, params)
    a.fista_step(3)  # progress that the restore must discard
    a.fista_restore(state)
    a.fista_step(10)
    assert torch.equal(straight, a.fista_get())
    assert a.refine_stats()[0] == 20
    a.close()
    if prec == "fp32":
        b = sw.Operator(g, K, s, precision=prec)
        b.fista_init(yd, params)
        b.fista_restore(state)
        b.fista_step(10)
        assert torch.equal(straight, b.fista_get())
        b.close()


def test_checkpoint_refuses_other_settings(tiny):
    g, s, K, y, alpha, _ = tiny
    yd = dev(y)
    a = sw.Operator(g, K, s)
    a.fista_init(yd, _params(alpha, 5))
    a.fista_step(2)
    state = a.fista_save()
    b = sw.Operator(g, K, s)
    b.fista_init(yd, sw.SolveParams(step=alpha, lambda_l1=2 * TINY.lam_l1,
                                    lambda_tv=TINY.lam_tv, inner_iters=TINY.inner, max_iters=5))
    with pytest.raises(sw.SwoptError):
        b.fista_restore(state)
    with pytest.raises(sw.SwoptError):
        b.fista_restore(state[:100])
    a.close()
    b.close()


def test_tv_barrier_timeout_is_reported_and_the_handle_recovers(tiny):
    """Failure detection without a GPU fault: the test hook makes every grid
    barrier of the cooperative TV prox wait for a block that does not exist;
    each wait gives up after its poll limit, the kernel returns, and
    check_device reports a timeout.  With the hook cleared the same handle
    computes the prox correctly again."""
    g, s, K, _, _, _ = tiny
    op = sw.Operator(g, K, s)
    z = synth.gaussian(g.c_shape(), 31) * 0.1
    zd = dev(z)
    ok = op.prox_tv(zd, 0.05, 10)
    op.check_device()
    op.debug_barrier(phantom_arrivals=1, poll_limit=1 << 14)
    op.prox_tv(zd, 0.05, 10)
    with pytest.raises(sw.SwoptError) as e:
        op.check_device()
    assert e.value.status == 5  # SWOPT_ERR_TIMEOUT
    op.debug_barrier(0, 0)
    again = op.prox_tv(zd, 0.05, 10)
    op.check_device()
    assert torch.equal(again, ok)
    assert rel(host(again), oracle.prox_tv(z, 0.05, 10)) <= 1e-5
    op.close()
