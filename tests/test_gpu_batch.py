"""Ragged batches (hermite_batch_*): every problem of a mixed batch matches an
individual context and the oracle; graph replay equals direct launches; the
autotuner returns a working configuration."""
import numpy as np
import pytest

from tests.gpu_util import lib_built, need_gpu, rel_l2, run_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


def _mixed(d, seed, n):
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(n):
        N = int(rng.choice([3, 5, 8, 13] if d < 3 else [3, 4, 6]))
        m = int(rng.choice([1, 2, 3] if d == 3 else [2, 3, 4, 6]))
        variant = int(rng.integers(0, 3))
        bc = int(rng.integers(0, 3))
        lam = float(rng.uniform(0.5, 1.0))
        h = 1.0 / N
        probs.append((d, m, N, 1.0, h, lam * h, variant, bc))
    return probs


def _states(hb, batch, seed):
    rng = np.random.default_rng(seed)
    out = []
    for g in batch.problems:
        n0 = g.nodes(0)
        u = rng.standard_normal((n0, g.Nu))
        v = rng.standard_normal((n0, g.Nv))
        g.set_state(u, v)
        out.append((u, v))
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_batch_matches_single_contexts_and_oracle(hb, orc, d, precision):
    import torch

    probs = _mixed(d, 10 + d, 10 if d < 3 else 6)
    batch = hb.HermiteBatch(probs, precision=precision)
    s = torch.cuda.Stream()
    batch.set_stream(s)
    init = _states(hb, batch, 3)
    batch.step(3)
    for p, (prob, (u, v)) in enumerate(zip(probs, init)):
        g = batch.problem(p)
        bu, bv = g.get_state()
        single = hb.Hermite(*prob, precision=precision)
        single.set_state(u, v)
        single.step(3)
        su, sv = single.get_state()
        assert rel_l2(bu, su) <= 1e-13, (p, prob)
        P = orc.Problem(*prob)
        tol = run_tol(prob[1], 1e-11 if precision == 0 else 1e-10)
        if prob[6] == orc.CONSERVATIVE:
            ou, _ = P.run(u, nsteps=3, dual_u=P.cons_start(u, v if prob[1] >= 1 else None))
            assert rel_l2(bu, ou) <= tol, (p, prob)
        else:
            ou, ov = P.run(u, v, nsteps=3)
            assert rel_l2(np.concatenate([bu, bv], 1), np.concatenate([ou, ov], 1)) <= tol, (p, prob)
    batch.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_direct_launches(hb, precision):
    import torch

    probs = _mixed(2, 5, 8)
    outs = []
    for stream in (torch.cuda.Stream(), None):
        batch = hb.HermiteBatch(probs, precision=precision)
        if stream is not None:
            batch.set_stream(stream)
        _states(hb, batch, 7)
        batch.step(4)
        outs.append([batch.problem(p).get_state()[0] for p in range(len(probs))])
        batch.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_autotune_and_config(hb):
    import torch

    probs = _mixed(2, 9, 12)
    batch = hb.HermiteBatch(probs, precision=1)
    batch.set_stream(torch.cuda.Stream())
    items, blocks, ms = batch.autotune()
    assert items in (256, 1024, 4096) and blocks in (1, 2, 4, 8) and ms > 0
    init = _states(hb, batch, 2)
    batch.step(2)
    u, _ = batch.problem(0).get_state()
    single = hb.Hermite(*probs[0], precision=1)
    single.set_state(*init[0])
    single.step(2)
    assert rel_l2(u, single.get_state()[0]) <= 1e-13
    batch.config(64, 3)
    batch.step(1)
    with pytest.raises(hb.HermiteError):
        batch.config(8, 1)
    batch.close()


def test_batch_rejects_mixed_dimensions_and_unequal_progress(hb):
    with pytest.raises(hb.HermiteError):
        hb.HermiteBatch([(1, 2, 8, 1.0, 0.125, 0.1, 0, 0), (2, 2, 8, 1.0, 0.125, 0.1, 0, 0)])
    batch = hb.HermiteBatch([(1, 2, 8, 1.0, 0.125, 0.1, 0, 0), (1, 3, 8, 1.0, 0.125, 0.1, 1, 0)])
    batch.problem(0).advance_half(1)
    with pytest.raises(hb.HermiteError) as e:
        batch.step(1)
    assert e.value.code == -6
    batch.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_state_transfer_matches_per_problem_calls(hb, precision):
    """hermite_batch_get/set_states_device move every problem's level in one
    launch, back to back, exactly like the per-problem calls."""
    import torch

    probs = [p for p in _mixed(2, 21, 9) if p[6] != 1]
    batch = hb.HermiteBatch(probs, precision=precision)
    batch.set_stream(torch.cuda.Stream())
    rng = np.random.default_rng(4)
    us, vs = [], []
    for g in batch.problems:
        n0 = g.nodes(0)
        us.append(rng.standard_normal((n0, g.Nu)))
        vs.append(rng.standard_normal((n0, g.Nv)))
    U = torch.as_tensor(np.concatenate([u.ravel() for u in us])).cuda()
    V = torch.as_tensor(np.concatenate([v.ravel() for v in vs])).cuda()
    batch.set_states_device(U, V)
    batch.step(2)
    U2, V2 = torch.empty_like(U), torch.empty_like(V)
    batch.get_states_device(0, U2, V2)
    torch.cuda.synchronize()
    ou, ov = 0, 0
    for p, (prob, u, v) in enumerate(zip(probs, us, vs)):
        g = batch.problem(p)
        gu, gv = g.get_state()
        assert np.array_equal(U2[ou:ou + gu.size].cpu().numpy().reshape(gu.shape), gu)
        assert np.array_equal(V2[ov:ov + gv.size].cpu().numpy().reshape(gv.shape), gv)
        single = hb.Hermite(*prob, precision=precision)
        single.set_state(u, v)
        single.step(2)
        assert rel_l2(gu, single.get_state()[0]) <= 1e-13
        ou += gu.size
        ov += gv.size
    cons = [p for p in _mixed(2, 21, 9) if p[6] == 1][:1]
    if cons:
        cb = hb.HermiteBatch(cons)
        with pytest.raises(hb.HermiteError) as e:
            cb.set_states_device(U, V)
        assert e.value.code == -6
        cb.close()
    batch.close()
