"""GPU tests of the grouped persistent launch (gtt_group_*) and the autotuner."""
import os

import numpy as np
import pytest
import torch

import gtt_inputs as gi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2507_02420_gb300 import build
    build.build()
    import paper_2507_02420_gb300 as g
    torch.cuda.set_device(0)
    return g


def up(a):
    a = np.asarray(a)
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def rel(a, ref):
    return float(np.linalg.norm(up(a) - ref) / max(np.linalg.norm(ref), 1e-300))


def make_requests(specs, seed):
    rng = np.random.default_rng(seed)
    reqs, host = [], []
    for b, n, dt, inv in specs:
        if dt == "c64":
            W = gi.haar_unitary(b, rng).astype(np.complex64)
            x = gi.complex_normal_x((b ** n,), rng, np.complex64)
        else:
            W = gi.haar_orthogonal(b, rng).astype(np.float32)
            x = gi.normal_x((b ** n,), rng, np.float32)
        xd = torch.from_numpy(x).cuda()
        reqs.append(dict(b=b, n=n, dtype=dt, W=W, x=xd, y=torch.empty_like(xd), inverse=inv))
        host.append((W, x))
    return reqs, host


def test_small_mixed_group_matches_oracle(g):
    rng = np.random.default_rng(8000)
    specs = []
    for i in range(60):
        b = int(rng.choice([2, 3, 4, 5, 6, 7, 8, 16]))
        nmax = {2: 16, 3: 10, 4: 8, 5: 6, 6: 6, 7: 5, 8: 5, 16: 4}[b]
        n = int(rng.integers(1, nmax + 1))
        specs.append((b, n, "c64" if i % 2 else "f32", bool(i % 5 == 0)))
    reqs, host = make_requests(specs, 8001)
    grp = g.Group(reqs)
    grp.execute()
    torch.cuda.synchronize()
    grp.check()
    for (b, n, dt, inv), rq, (W, x) in zip(specs, reqs, host):
        ref = oracle.adjoint(up(W), up(x)) if inv else oracle.modes(up(W), up(x))
        assert rel(rq["y"].cpu().numpy(), ref) <= 2e-6, (b, n, dt, inv)


@pytest.mark.parametrize("with_small", [False, True])
def test_large_requests_run_as_pass_chains(g, with_small):
    """Requests of 2 MiB or more run as chains of their shape's pass kernels on
    side streams of the group's graph (TMA, b = 8 tile and CUDA-core passes,
    forward and inverse, several requests sharing one shape with different W);
    a group of only such requests has no persistent-kernel work at all."""
    specs = [(4, 10, "c64", False), (4, 10, "c64", True), (8, 7, "f32", False), (2, 20, "f32", True),
             (16, 5, "c64", False), (3, 13, "f32", False)]
    if with_small:
        specs += [(4, 5, "c64", False), (5, 4, "f32", True), (2, 9, "f32", False)]
    reqs, host = make_requests(specs, 8050 + int(with_small))
    grp = g.Group(reqs)
    d = grp.describe()
    assert d["direct_requests"] == 6
    assert (d["work_items"] > 0) == with_small
    for _ in range(2):   # replays give the same result
        grp.execute()
        torch.cuda.synchronize()
        grp.check()
        for (b, n, dt, inv), rq, (W, x) in zip(specs, reqs, host):
            ref = oracle.adjoint(up(W), up(x)) if inv else oracle.modes(up(W), up(x))
            assert rel(rq["y"].cpu().numpy(), ref) <= 2e-6, (b, n, dt, inv)


def test_group_replay_is_repeatable_and_in_place(g):
    specs = [(4, 9, "c64", False), (2, 14, "f32", False), (16, 3, "f32", True), (3, 8, "c64", False)]
    reqs, host = make_requests(specs, 8100)
    grp = g.Group(reqs)
    grp.execute()
    first = [r["y"].clone() for r in reqs]
    grp.execute()
    torch.cuda.synchronize()
    grp.check()
    for a, r in zip(first, reqs):
        assert torch.equal(a, r["y"])
    # in place: y aliases x
    reqs2, host2 = make_requests(specs, 8101)
    for r in reqs2:
        r["y"] = r["x"]
    grp2 = g.Group(reqs2)
    grp2.execute()
    torch.cuda.synchronize()
    for (b, n, dt, inv), r, (W, x) in zip(specs, reqs2, host2):
        ref = oracle.adjoint(up(W), up(x)) if inv else oracle.modes(up(W), up(x))
        assert rel(r["x"].cpu().numpy(), ref) <= 2e-6


def test_grouped_1000_uneven_requests(g):
    """The uneven workload: 1000 requests, b in {2,3,4,5,8,16}, N log-uniform
    in [2^10, 2^22], FP32 / complex64, one persistent launch in a CUDA graph.
    Every request keeps its norm (unitary / orthogonal W); 40 sampled requests
    are compared with the oracle element by element."""
    rqs = gi.grouped_requests()
    reqs = []
    host = {}
    sample = set(range(0, 1000, 25))
    for i, r in enumerate(rqs):
        W, x = gi.request_inputs(r)
        xd = torch.from_numpy(x).cuda()
        reqs.append(dict(b=r.b, n=r.n, dtype=r.dtype, W=W, x=xd, y=torch.empty_like(xd)))
        if i in sample:
            host[i] = (W, x)
    grp = g.Group(reqs)
    d = grp.describe()
    grp.execute()
    torch.cuda.synchronize()
    grp.check()
    print("grouped:", d)
    for r in reqs:
        nx = torch.linalg.vector_norm(r["x"]).item()
        ny = torch.linalg.vector_norm(r["y"]).item()
        assert abs(ny / nx - 1) <= 1e-5
    for i, (W, x) in host.items():
        ref = oracle.modes(up(W), up(x))
        assert rel(reqs[i]["y"].cpu().numpy(), ref) <= 1e-5, (i, rqs[i])


def test_group_rejects_unsupported_requests(g):
    x = torch.zeros(9 ** 2, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GTTError) as ei:
        g.Group([dict(b=9, n=2, dtype="f32", W=np.eye(9, dtype=np.float32), x=x, y=x)])
    assert ei.value.status == 2
    y = torch.zeros(64, dtype=torch.complex128, device="cuda")
    with pytest.raises(g.GTTError):
        g.Group([dict(b=2, n=6, dtype="c128", W=np.eye(2), x=y, y=y)])


def test_autotune_picks_a_correct_schedule_and_caches_it(g, tmp_path):
    rng = np.random.default_rng(8200)
    W = gi.haar_unitary(4, rng).astype(np.complex64)
    x = gi.complex_normal_x((1, 4 ** 10), rng, np.complex64)
    plan = g.Plan(W, 10, "c64", 1)
    plan.autotune(48)
    d = plan.describe()
    y = plan.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), oracle.modes(up(W), up(x))) <= 2e-6
    path = str(tmp_path / "tune.json")
    g.autotune_cache_save(path)
    text = open(path).read()
    assert '"digits"' in text and "|b4|n10|" in text
    g.autotune_cache_load(path)
    plan2 = g.Plan(W, 10, "c64", 1)   # a new plan picks the cached schedule
    assert [p["g"] for p in plan2.describe()["passes"]] == [p["g"] for p in d["passes"]]


def test_explicit_schedule_and_rejections(g):
    rng = np.random.default_rng(8300)
    W = gi.haar_orthogonal(8, rng).astype(np.float32)
    x = gi.normal_x((2, 8 ** 6), rng, np.float32)
    plan = g.Plan(W, 6, "f32", 2)
    ref = oracle.modes(up(W), up(x))
    # (a first-pass run k > 1 means tiles of k consecutive blocks of 8^digits[0])
    for digits, runs in (([3, 3], [1, 64]), ([2, 2, 2], [1, 8, 64]), ([5, 1], [1, 8]),
                         ([1] * 6, [1, 8, 8, 8, 8, 8]), ([3, 3], [2, 64]), ([2, 4], [8, 8])):
        plan.set_passes(digits, runs)
        y = plan.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), ref) <= 2e-6, digits
    # digits not summing to n, first-pass blocks not dividing the data, a run
    # not dividing b^m0, a 1 MiB tile
    for digits, runs in (([3, 2], [1, 8]), ([3, 3], [3, 8]), ([3, 3], [1, 7]), ([6], [1])):
        with pytest.raises(g.GTTError):
            plan.set_passes(digits, runs)
