"""GPU parity of the learned Newton predictor kernels (tvi_predictor_forward,
tvi_predictor_train_step) with the FP64 reference in oracle/predictor.py, and
the predictor's use as Newton's starting guess inside tvi_integrate.

The kernels compute in FP32.  A dot product of K <= 256 terms carries a
relative error of order K * 2^-24 ~ 1.5e-5 of the sum of |terms|; the gates
below (1e-4 of the largest magnitude of each compared quantity) leave margin
for that and for the two stacked layers, while a wrong index, a dropped term
or a transposed operand moves results by O(1).
"""
import numpy as np
import pytest

import workloads
from oracle import predictor as OP
from parity_helpers import be_step_bound, be_step_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B1, B2 = 0.9, 0.999


@pytest.fixture(scope="module")
def tvi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_08649_gb300 as tvi
    from paper_2310_08649_gb300 import build
    build.build()
    return tvi


def random_predictor(seed, n_in, hid, n_out):
    """Packed vector with Xavier-scaled weights and positive std / scale."""
    off, total = OP.layout(n_in, hid, n_out)
    g = np.random.Generator(np.random.PCG64(seed))
    p = np.zeros(total)

    def put(name, v):
        a, s = off[name]
        p[a:a + s] = v

    put("mean", g.standard_normal(n_in))
    put("std", g.uniform(0.5, 2.0, n_in))
    put("scale", g.uniform(0.5, 2.0, n_out))
    for W, fi, fo in (("W1", n_in, hid), ("W2", hid, hid), ("W3", hid, n_out)):
        a = np.sqrt(6.0 / (fi + fo))
        put(W, g.uniform(-a, a, fi * fo))
    for b, k in (("b1", hid), ("b2", hid), ("b3", n_out)):
        put(b, 0.1 * g.standard_normal(k))
    return p.astype(np.float32)


def f32dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def make_pred(tvi, dims, packed):
    from paper_2310_08649_gb300.predictor import Predictor, PredictorSpec
    n_in, hid, n_out = dims
    spec = PredictorSpec(chunk=n_out // 2, hidden=hid)
    assert spec.n_in == n_in
    P = Predictor(spec, seed=0)
    P.packed.copy_(f32dev(packed))
    return P


DIMS = [(5, 6, 4), (103, 256, 200)]  # (3 + c, H, 2 c) with c = 2 and c = 100


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("M", [1, 37, 300])
def test_inference_parity(tvi, dims, M):
    packed = random_predictor(11, *dims)
    x = np.random.Generator(np.random.PCG64(12)).standard_normal((M, dims[0])).astype(np.float32)
    P = make_pred(tvi, dims, packed)
    y = P.forward(f32dev(x)).cpu().numpy()
    ref = OP.forward(packed.astype(np.float64), *dims, x.astype(np.float64))
    assert np.abs(y - ref).max() <= 1e-4 * np.abs(ref).max()


def test_inference_empty_batch(tvi):
    P = make_pred(tvi, DIMS[0], random_predictor(1, *DIMS[0]))
    assert P.forward(torch.empty((0, 5), dtype=torch.float32, device="cuda")).shape == (0, 4)


def segments(dims):
    off, _ = OP.layout(*dims)
    begin = off["W1"][0]
    return {k: (a - begin, s) for k, (a, s) in off.items() if a >= begin}


def close_per_segment(a, b, dims, rel):
    for name, (o, s) in segments(dims).items():
        ref = b[o:o + s]
        err = np.abs(a[o:o + s] - ref).max()
        assert err <= rel * max(np.abs(ref).max(), 1e-30), (name, err, np.abs(ref).max())


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("M", [37, 256])
def test_train_step_parity(tvi, dims, M):
    """Two Adam steps on different batches.  After step 1 from zero moments,
    m = (1 - beta1) g exposes the FP32 gradient, compared with the reference
    gradient segment by segment; after step 2 both moments and the weights are
    compared with two reference steps."""
    n_in, hid, n_out = dims
    packed = random_predictor(21, *dims)
    off, _ = OP.layout(*dims)
    g = np.random.Generator(np.random.PCG64(22))
    S = 2 * M
    x = g.standard_normal((S, n_in)).astype(np.float32)
    sc = packed[off["scale"][0]:off["scale"][0] + n_out]
    t = (g.standard_normal((S, n_out)) * sc).astype(np.float32)
    P = make_pred(tvi, dims, packed)
    xd, td = f32dev(x), f32dev(t)
    rows1 = torch.arange(0, M, dtype=torch.int32, device="cuda")
    rows2 = torch.arange(M, S, dtype=torch.int32, device="cuda")
    lr = 1e-3

    loss1 = P.train_step(xd, td, lr, rows1).cpu().numpy()[0]
    m1 = P.m.cpu().numpy().astype(np.float64)
    v1 = P.v.cpu().numpy().astype(np.float64)
    p64 = packed.astype(np.float64)
    n = m1.size
    rp1, rm1, rv1, rloss1 = OP.train_step(p64, np.zeros(n), np.zeros(n), *dims,
                                          x[:M].astype(np.float64), t[:M].astype(np.float64),
                                          lr, 1)
    assert abs(loss1 - rloss1) <= 1e-4 * rloss1
    grad_gpu = m1 / float(np.float32(1) - np.float32(B1))
    close_per_segment(grad_gpu, rm1 / (1 - B1), dims, 1e-4)
    close_per_segment(v1, rv1, dims, 3e-4)
    # step 1 moves each weight by lr * sign(g) where |g| is well above the FP32 error
    p1 = P.packed.cpu().numpy().astype(np.float64)
    begin = off["W1"][0]
    assert np.array_equal(p1[:begin], p64[:begin])  # normalisation is not trained
    gref = rm1 / (1 - B1)
    big = np.abs(gref) > 1e-2 * np.abs(gref).max()
    step = (p1 - p64)[begin:][big]
    assert np.allclose(step, (rp1 - p64)[begin:][big], rtol=2e-3, atol=0)

    loss2 = P.train_step(xd, td, lr, rows2).cpu().numpy()[0]
    rp2, rm2, rv2, rloss2 = OP.train_step(rp1, rm1, rv1, *dims, x[M:].astype(np.float64),
                                          t[M:].astype(np.float64), lr, 2)
    assert abs(loss2 - rloss2) <= 1e-4 * rloss2
    close_per_segment(P.m.cpu().numpy().astype(np.float64), rm2, dims, 3e-4)
    close_per_segment(P.v.cpu().numpy().astype(np.float64), rv2, dims, 1e-3)
    p2 = P.packed.cpu().numpy().astype(np.float64)
    assert np.abs(p2 - rp2).max() <= 4 * lr  # Adam steps are bounded by lr each


def test_row_gather_is_bitwise_identical(tvi):
    """A batch named by row indices trains exactly like the same rows copied out."""
    dims = DIMS[1]
    packed = random_predictor(31, *dims)
    g = np.random.Generator(np.random.PCG64(32))
    x = g.standard_normal((500, dims[0])).astype(np.float32)
    t = g.standard_normal((500, dims[2])).astype(np.float32)
    rows = g.permutation(500)[:130].astype(np.int32)
    A = make_pred(tvi, dims, packed)
    Bp = make_pred(tvi, dims, packed)
    la = A.train_step(f32dev(x), f32dev(t), 1e-3, torch.as_tensor(rows, device="cuda"))
    lb = Bp.train_step(f32dev(x[rows]), f32dev(t[rows]), 1e-3)
    assert torch.equal(la, lb)
    assert torch.equal(A.packed, Bp.packed)
    assert torch.equal(A.m, Bp.m) and torch.equal(A.v, Bp.v)


def test_train_step_rejects_bad_arguments(tvi):
    from paper_2310_08649_gb300 import _lib
    P = make_pred(tvi, DIMS[0], random_predictor(1, *DIMS[0]))
    x = torch.zeros((4, 5), dtype=torch.float32, device="cuda")
    t = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(_lib.TviError) as e:
        P.train_step(x, t, 1e-3, workspace=small)
    assert e.value.code == -2  # TVI_EWORKSPACE


# ---------------------------------------------------------------------------
# The predictor inside tvi_integrate (van der Pol, chunk 100).
# ---------------------------------------------------------------------------
def vdp_run(tvi, w, precision, tol, pred=None):
    m = tvi.Model.from_spec(w["spec"])
    extra = pred.options() if pred is not None else {}
    o = tvi.Options(chunk=100, tol_abs=tol, precision=precision, **extra)
    d = {k: torch.as_tensor(w[k], dtype=torch.float64, device="cuda")
         for k in ("y0", "times", "params")}
    y, stats, st, rc = tvi.integrate(m, o, d["y0"], d["times"], d["params"],
                                     raise_on_status=False)
    torch.cuda.synchronize()
    return y.cpu().numpy(), stats.cpu().numpy(), st.cpu().numpy(), rc


@pytest.mark.parametrize("kind", ["huge", "nan"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_useless_predictor_is_always_rejected(tvi, kind, precision):
    """A predictor whose guesses are far off (or not finite) loses every residual
    comparison, so the integration is bit-for-bit the dy = 0 one."""
    dims = (103, 16, 200)
    packed = random_predictor(41, *dims)
    off, _ = OP.layout(*dims)
    a, s = off["scale"] if kind == "huge" else off["b3"]
    packed[a:a + s] = 1e8 if kind == "huge" else np.nan
    P = make_pred(tvi, dims, packed)
    w = workloads.vdp(B=16, N=2000)
    y0, s0, st0, rc0 = vdp_run(tvi, w, precision, 1e-8)
    y1, s1, st1, rc1 = vdp_run(tvi, w, precision, 1e-8, P)
    assert rc0 == 0 and rc1 == 0
    assert np.array_equal(y0, y1)
    assert np.array_equal(s0[:, :4], s1[:, :4])
    assert not s1[:, 4].any()
    assert s1[:, 5].sum() > 0
    # with every guess rejected, the back-off tries chunks 0, 2, 6, 14, ... (gaps
    # 2^k - 1, k <= 5): exactly that many guesses where no chunk was halved
    clean = s1[:, 2] == 0  # no halving: every attempt had the predictor's length
    expect = []
    for chunks in s1[clean, 1]:
        tries, nxt, k = 0, 0, 0
        for i in range(chunks):
            if i == nxt:
                tries += 1
                k = min(k + 1, 5)
                nxt = i + 2 ** k
        expect.append(tries)
    assert np.array_equal(s1[clean, 5], np.array(expect))


def test_predictor_option_validation(tvi):
    from paper_2310_08649_gb300 import _lib
    dims = (103, 16, 200)
    P = make_pred(tvi, dims, random_predictor(1, *dims))
    w = workloads.linear_stiff(B=2, N=200)
    m = tvi.Model.from_spec(w["spec"])
    d = {k: torch.as_tensor(w[k], dtype=torch.float64, device="cuda")
         for k in ("y0", "times", "params")}
    with pytest.raises(_lib.TviError) as e:  # the predictor is built for van der Pol only
        tvi.integrate(m, tvi.Options(chunk=100, **P.options()), d["y0"], d["times"], d["params"])
    assert e.value.code == -7
    wv = workloads.vdp(B=2, N=200)
    mv = tvi.Model.from_spec(wv["spec"])
    dv = {k: torch.as_tensor(wv[k], dtype=torch.float64, device="cuda")
          for k in ("y0", "times", "params")}
    for chunk, hid in ((129, 16), (100, 15), (100, 258)):
        o = tvi.Options(chunk=100, predictor=P.packed, predictor_chunk=chunk,
                        predictor_hidden=hid)
        with pytest.raises(_lib.TviError) as e:
            tvi.integrate(mv, o, dv["y0"], dv["times"], dv["params"])
        assert e.value.code == -1


def test_trained_predictor_keeps_results(tvi, oracle_lib):
    """Train on solver chunks of training seeds, integrate a held-out seed: the
    predictor wins some residual comparisons, every step still solves backward
    Euler to the tolerance (checked step by step), and the trajectory agrees with the dy = 0 run within
    the forward error that stopping Newton at tol allows."""
    from oracle import Model as OModel
    from paper_2310_08649_gb300.predictor import Predictor, PredictorSpec, solver_dataset
    spec = PredictorSpec()
    x, t = solver_dataset(lambda s: workloads.vdp(seed=s, B=64), range(3000, 3004), spec)
    P = Predictor(spec, seed=0)
    P.set_normalisation(x, t)
    losses = P.fit(x, t, epochs=60, batch=512, lr=1e-3, lr_end=1e-5, seed=1)
    assert losses[-1] < 0.5 * losses[0]
    tol = 1e-8
    w = workloads.vdp(seed=4000)
    y0, s0, st0, rc0 = vdp_run(tvi, w, "fp32", tol)
    y1, s1, st1, rc1 = vdp_run(tvi, w, "fp32", tol, P)
    assert rc0 == 0 and rc1 == 0 and not st1.any()
    assert s1[:, 4].sum() > 0
    m = OModel.from_spec(w["spec"])
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], y0, tol)
    scale = np.abs(y0).max(axis=(1, 2))
    err = np.abs(y1 - y0).max(axis=(1, 2)) / scale
    bad = np.nonzero(err > np.maximum(1e-5, 20.0 * est))[0]
    assert bad.size == 0, (bad, err[bad], est[bad])
    # every step against the oracle's solve of that step from the run's own y_{k-1}:
    # residuals of tol leave at most be_step_bound (one step's conditioning)
    step = be_step_errors(oracle_lib, m, w, y1)
    assert np.all(step <= be_step_bound(oracle_lib, m, w, y1, tol)), step.max()
