"""GPU parity of plan groups (uw_group_*): many independent products of
uneven sizes issued as one unit over internal streams, tuned per plan, and
captured into one CUDA graph; compared with the dense oracle and with the
plans' own calls."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, wavelets as W
from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, F64, PERIODIC, VMP, Plan, PlanGroup, build, inputs

pytestmark = pytest.mark.gpu
TOL = {F64: 1e-12, F32: 1e-5, F32_SPLIT_BF16: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def uneven_instances(rng, n, Rs, qs, ps):
    """Instance shapes drawn like the batched uneven workload: R, q, p,
    boundary, level decay alpha in [1, 2] and a 10-40% radial multilevel mask."""
    out = []
    for _ in range(n):
        p = int(rng.choice(ps))
        R = int(rng.choice([r for r in Rs if r >= W.default_J0(p) + 1]))
        q = int(rng.choice(qs))
        bd = int(rng.choice([PERIODIC, VMP]))
        N = 2 ** (R + q)
        omega = inputs.mask_2d(rng, N, float(rng.uniform(0.1, 0.4)))
        x = inputs.coeffs_2d(rng, R, W.default_J0(p), float(rng.uniform(1.0, 2.0)))
        out.append((R, q, p, bd, omega, x))
    return out


def tensors(plans, xs, ys, dt):
    xd = [torch.tensor(x, dtype=dt, device="cuda") for x in xs]
    yd = [torch.tensor(y, dtype=dt, device="cuda") for y in ys]
    yo = [torch.empty(pl.m, dtype=dt, device="cuda") for pl in plans]
    xo = [torch.empty_like(x) for x in xd]
    return xd, yd, yo, xo


@pytest.mark.parametrize("prec", [F32, F64, F32_SPLIT_BF16])
def test_group_uneven_against_dense_oracle(prec):
    rng = np.random.default_rng(3)
    inst = uneven_instances(rng, 10, Rs=(6, 7), qs=(1, 2), ps=(1, 2, 4, 6, 8))
    plans = [Plan(2, R, q, p, bd, omega=om) for R, q, p, bd, om, _ in inst]
    xs = [x for *_, x in inst]
    ys = [rng.standard_normal(pl.m) for pl in plans]
    want_y, want_x = [], []
    for (R, q, p, bd, om, x), y in zip(inst, ys):
        G = dense.G1d(R, q, p, bd)
        want_y.append(dense.forward2d(x, R, q, p, bd, W.default_J0(p), om, G=G))
        want_x.append(dense.adjoint2d(y, R, q, p, bd, W.default_J0(p), om, G=G))
    dt = torch.float64 if prec == F64 else torch.float32
    group = PlanGroup(plans, nstreams=4)
    xd, yd, yo, xo = tensors(plans, xs, ys, dt)
    group.forward(xd, yo, prec)
    group.adjoint(yd, xo, prec)
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert rel(yo[i].cpu().numpy(), want_y[i]) < TOL[prec], i
        assert rel(xo[i].cpu().numpy(), want_x[i]) < TOL[prec], i
    # tuning chooses a variant per plan; results stay within the tolerance
    group.tune([x.clone() for x in xd], [torch.empty_like(y) for y in yo], prec, reps=2)
    group.forward(xd, yo, prec)
    group.adjoint(yd, xo, prec)
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert rel(yo[i].cpu().numpy(), want_y[i]) < TOL[prec], i
        assert rel(xo[i].cpu().numpy(), want_x[i]) < TOL[prec], i
    group.close()


def test_group_graph_capture_matches_plain_calls():
    """64 uneven instances (R in 6..9, q in 1..2, p in {1,2,4,6,8}): the group's
    pair captured as one CUDA graph and replayed twice equals each plan's own
    forward and adjoint; plans get their fused coarse launches back after the
    group is closed."""
    rng = np.random.default_rng(33)
    inst = uneven_instances(rng, 64, Rs=(6, 7, 8, 9), qs=(1, 2), ps=(1, 2, 4, 6, 8))
    plans = [Plan(2, R, q, p, bd, omega=om) for R, q, p, bd, om, _ in inst]
    xs = [x for *_, x in inst]
    ys = [rng.standard_normal(pl.m) for pl in plans]
    xd, yd, yo, xo = tensors(plans, xs, ys, torch.float32)
    ref_y = [pl.forward(x, precision=F32) for pl, x in zip(plans, xd)]
    ref_x = [pl.adjoint(y, precision=F32) for pl, y in zip(plans, yd)]
    torch.cuda.synchronize()
    group = PlanGroup(plans, nstreams=8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        group.forward(xd, yo, F32)        # first calls outside capture (one-time setup)
        group.adjoint(yd, xo, F32)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        group.forward(xd, yo, F32, stream=s)
        group.adjoint(yd, xo, F32, stream=s)
    for _ in range(2):
        for t in yo + xo:
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for i in range(len(plans)):
            # the group runs the coarse levels per level (generic tiles); the
            # plans' own calls use the fused register-window tiles
            assert rel(yo[i].cpu().numpy(), ref_y[i].cpu().numpy()) < 1e-6, i
            assert rel(xo[i].cpu().numpy(), ref_x[i].cpu().numpy()) < 1e-6, i
    group.close()
    again = plans[-1].forward(xd[-1], precision=F32)
    torch.cuda.synchronize()
    assert rel(again.cpu().numpy(), ref_y[-1].cpu().numpy()) == 0.0


def test_group_rejects_a_plan_twice_and_a_plan_in_two_groups():
    """A plan owns one workspace: the same plan on two internal streams, or in
    two live groups, would race on it.  Both are refused at creation; after
    the first group is destroyed the plan may join another."""
    from paper_2106_00554_gb300 import UWError
    a = Plan(2, 6, 1, 2, VMP)
    b = Plan(2, 6, 1, 4, PERIODIC)
    with pytest.raises(UWError) as e:
        PlanGroup([a, b, a], nstreams=2)
    assert e.value.status == 1
    g = PlanGroup([a, b], nstreams=2)
    with pytest.raises(UWError) as e:
        PlanGroup([b], nstreams=1)
    assert e.value.status == 1
    g.close()
    g2 = PlanGroup([b], nstreams=1)
    g2.close()
    a.close()
    b.close()


def _group_case(seed, n):
    rng = np.random.default_rng(seed)
    inst = uneven_instances(rng, n, Rs=(6, 7, 8), qs=(1, 2), ps=(1, 2, 4, 6, 8))
    plans = [Plan(2, R, q, p, bd, omega=om) for R, q, p, bd, om, _ in inst]
    xs = [x for *_, x in inst]
    ys = [rng.standard_normal(pl.m) for pl in plans]
    return inst, plans, xs, ys


def test_persistent_group_launch_matches_the_forked_streams(monkeypatch):
    """FP32 products of a group of 2D plans run as one persistent launch (a
    grid draining a queue of (instance, phase, items) tasks).  The results
    equal the forked-stream path within FP32 rounding and the dense oracle
    within 1e-5; the launch is in use before any tuning."""
    inst, plans, xs, ys = _group_case(41, 24)
    xd, yd, yo, xo = tensors(plans, xs, ys, torch.float32)
    group = PlanGroup(plans, nstreams=4)
    prm = group.params()
    assert prm["persistent_available"] == 1 and prm["persistent_in_use"] == 1, prm
    group.forward(xd, yo, F32)
    group.adjoint(yd, xo, F32)
    torch.cuda.synchronize()
    got_y = [t.cpu().numpy() for t in yo]
    got_x = [t.cpu().numpy() for t in xo]
    monkeypatch.setenv("UW_GROUP_STREAMS", "1")
    group.forward(xd, yo, F32)
    group.adjoint(yd, xo, F32)
    torch.cuda.synchronize()
    monkeypatch.delenv("UW_GROUP_STREAMS")
    for i, (R, q, p, bd, om, x) in enumerate(inst):
        assert rel(got_y[i], yo[i].cpu().numpy()) < 1e-6, i
        assert rel(got_x[i], xo[i].cpu().numpy()) < 1e-6, i
        G = dense.G1d(R, q, p, bd)
        J0 = W.default_J0(p)
        assert rel(got_y[i], dense.forward2d(x, R, q, p, bd, J0, om, G=G)) < 1e-5, i
        assert rel(got_x[i], dense.adjoint2d(ys[i], R, q, p, bd, J0, om, G=G)) < 1e-5, i
    assert group.device_status() == 0
    group.close()


def test_persistent_group_wait_gives_up_and_reports(monkeypatch):
    """With a spin limit of zero every task whose previous phase is not yet
    complete gives up at once: the launch returns (no hang), the group reports
    UW_ERR_TIMEOUT and clears it, and the next call with the default limit is
    right."""
    inst, plans, xs, ys = _group_case(42, 12)
    xd, yd, yo, xo = tensors(plans, xs, ys, torch.float32)
    group = PlanGroup(plans, nstreams=2)
    group.forward(xd, yo, F32)
    torch.cuda.synchronize()
    want = [t.cpu().numpy().copy() for t in yo]
    monkeypatch.setenv("UW_GROUP_SPIN_LIMIT", "0")
    for t in yo:
        t.zero_()
    group.forward(xd, yo, F32)
    assert group.device_status() == 5
    monkeypatch.delenv("UW_GROUP_SPIN_LIMIT")
    group.forward(xd, yo, F32)
    assert group.device_status() == 0
    for i in range(len(plans)):
        assert rel(yo[i].cpu().numpy(), want[i]) == 0.0, i
    group.close()


def test_group_tuner_writes_and_reads_its_cache(tmp_path):
    """The tuner times the persistent launch's parameters and the forked
    streams, keeps the fastest, and records the choice in a JSON cache keyed by
    GPU, dimension, the instances' N and precision; a second tuning of a group
    of the same shape reads it back without timing."""
    import json
    inst, plans, xs, ys = _group_case(43, 8)
    xd, yd, yo, xo = tensors(plans, xs, ys, torch.float32)
    cache = str(tmp_path / "tune.json")
    group = PlanGroup(plans, nstreams=2)
    group.tune([x.clone() for x in xd], [torch.empty_like(y) for y in yo], F32, reps=1, cache=cache)
    first = group.params()
    group.close()
    entries = json.load(open(cache))
    assert len(entries) == 1
    (key, val), = entries.items()
    assert "|d2|" in key and len(val) == 6
    assert val[:5] == [first[k] for k in ("lines_per_task", "cols_per_task", "tiles_per_task", "radix",
                                          "ctas_per_sm")]
    group2 = PlanGroup(plans, nstreams=2)
    group2.tune([x.clone() for x in xd], [torch.empty_like(y) for y in yo], F32, reps=1, cache=cache)
    assert group2.params() == first
    group2.forward(xd, yo, F32)
    torch.cuda.synchronize()
    for i, (R, q, p, bd, om, x) in enumerate(inst):
        G = dense.G1d(R, q, p, bd)
        assert rel(yo[i].cpu().numpy(), dense.forward2d(x, R, q, p, bd, W.default_J0(p), om, G=G)) < 1e-5, i
    group2.close()
