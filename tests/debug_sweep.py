"""Small-case sweep run against the debug build (GTT_LIBRARY=debug):
every kernel family on small shapes -- all bases, n <= 6, odd batches, every
dtype -- with the plan's status word checked after each call.  Run as a
child process by tests/test_gpu_debug_build.py; prints one line per case and
exits non-zero on the first failed index check or wrong result."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import gtt_inputs as gi  # noqa: E402
import oracle  # noqa: E402
from paper_2507_02420_gb300 import _lib  # noqa: E402

assert _lib.DEBUG and _lib.LIB_PATH.endswith("libgtt_debug.so"), _lib.LIB_PATH
import paper_2507_02420_gb300 as g  # noqa: E402

TOL = {"f32": 2e-6, "c64": 2e-6, "f64": 1e-12, "c128": 1e-12}
NP = {"f32": np.float32, "c64": np.complex64, "f64": np.float64, "c128": np.complex128}


def up(a):
    a = np.asarray(a)
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def rel(a, ref):
    return float(np.linalg.norm(up(a) - ref) / max(np.linalg.norm(ref), 1e-300))


def make(b, n, batch, dt, rng):
    cplx = dt in ("c64", "c128")
    W = (gi.haar_unitary(b, rng) if cplx else gi.haar_orthogonal(b, rng)).astype(NP[dt])
    x = (gi.complex_normal_x((batch, b ** n), rng, np.complex128) if cplx
         else gi.normal_x((batch, b ** n), rng, np.float64)).astype(NP[dt])
    return W, x


def main():
    torch.cuda.set_device(0)
    rng = np.random.default_rng(20251)
    cases = 0
    for b in (2, 3, 4, 5, 7, 8, 16):
        for n in range(1, 7):
            if b ** n > (1 << 20):
                continue
            for dt in ("f32", "c64", "f64", "c128"):
                for batch in (1, 3):
                    W, x = make(b, n, batch, dt, rng)
                    plan = g.Plan(W, n, dt, batch)
                    xd = torch.from_numpy(x).cuda()
                    y = plan.forward(xd)
                    z = plan.inverse(y)
                    try:
                        plan.backward(xd, y)
                    except g.GTTError as e:  # a backward this shape does not have
                        assert e.status == 2, e
                    torch.cuda.synchronize()
                    plan.check()   # raises GTTError on a failed index check
                    ref = oracle.modes(up(W), up(x))
                    assert rel(y.cpu().numpy(), ref) <= TOL[dt], (b, n, dt, batch)
                    assert rel(z.cpu().numpy(), up(x)) <= 2 * TOL[dt], (b, n, dt, batch)
                    cases += 1
    # integer, precisions of the tensor-core paths, mixed radices, grouped launch
    xi = rng.integers(-2 ** 15, 2 ** 15, size=(3, 2 ** 6)).astype(np.int32)
    pi = g.Plan(np.array([[1, 1], [1, -1]], dtype=np.int32), 6, "i32", 3)
    pi.forward(torch.from_numpy(xi).cuda())
    pi.check()
    for prec in (g.PREC_BF16X3, g.PREC_BF16X2, g.PREC_TF32X3):
        for n in (3, 4, 5):
            W, x = make(16, n, 3, "f32", rng)
            plan = g.Plan(W, n, "f32", 3)
            plan.set_precision(prec)
            y = plan.forward(torch.from_numpy(x).cuda())
            plan.inverse(y)
            plan.check()
            assert rel(y.cpu().numpy(), oracle.modes(up(W), up(x))) <= 1e-4
            cases += 1
    W, x = make(4, 7, 3, "c64", rng)
    plan = g.Plan(W, 7, "c64", 3)
    plan.set_precision(g.PREC_TF32X3)
    y = plan.forward(torch.from_numpy(x).cuda())
    plan.inverse(y)
    plan.check()
    assert rel(y.cpu().numpy(), oracle.modes(up(W), up(x))) <= 1e-5
    radices = [3, 5, 2, 2, 7]
    Ws = [gi.haar_unitary(r, rng).astype(np.complex64) for r in radices]
    xm = gi.complex_normal_x((3, int(np.prod(radices))), rng, np.complex64)
    pm = g.Plan.mixed(Ws, "c64", 3)
    ym = pm.forward(torch.from_numpy(xm).cuda())
    pm.check()
    assert rel(ym.cpu().numpy(), oracle.modes_mixed([up(W) for W in Ws], up(xm))) <= 2e-6
    reqs = []
    for r in gi.grouped_requests(24):
        Wr, xr = gi.request_inputs(r)
        xd = torch.from_numpy(xr).cuda()
        reqs.append(dict(b=r.b, n=r.n, dtype=r.dtype, W=Wr, x=xd, y=torch.empty_like(xd)))
    grp = g.Group(reqs)
    grp.execute()
    torch.cuda.synchronize()
    grp.check()
    for q in reqs[:6]:
        assert rel(q["y"].cpu().numpy(), oracle.modes(up(q["W"]), up(q["x"].cpu().numpy()))) <= 2e-6
    print(f"debug sweep: {cases} single-base cases, integer, tensor-core, mixed and grouped runs: status clear")


if __name__ == "__main__":
    main()
