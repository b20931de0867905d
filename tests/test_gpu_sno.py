"""The surrogate's CUDA forward and backward passes against the FP64 CPU
reference (oracle/sno.py), training on GE data, and the GE fallback.

Tolerances: split mode (two-part BF16 operands) is accurate to about FP32, so
the prediction must match to 1e-4 relative L2 per problem and every
parameter block's gradient to 2e-3 relative L2; plain BF16 operands (unit
roundoff 2^-8 per operand) to 3e-2."""
import numpy as np
import pytest
import torch

from oracle import sno as S
from paper_1310_3422_gb300 import binding as B
from paper_1310_3422_gb300 import inputs
from paper_1310_3422_gb300 import surrogate as SG

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

SMALL = S.Arch(n=64, width=16, modes=8, layers=2, hidden=32)
FULL = S.Arch(n=1024, width=64, modes=16, layers=4, hidden=128)


def make_model(a: S.Arch, max_batch: int, seed: int = 1, split: int = 1):
    m = B.ge_sno_create(a.n, a.width, a.modes, a.layers, a.hidden, max_batch, seed)
    B.ge_sno_set_precision(m, split)
    return m


def get_params(m) -> np.ndarray:
    p = torch.empty(B.ge_sno_num_params(m), dtype=torch.float32, device=DEV)
    B.ge_sno_get_params(m, p)
    torch.cuda.synchronize()
    return p.cpu().numpy()


def problem_batch(a: S.Arch, batch: int, seed: int):
    pr = inputs.surrogate_problems(batch, a.n, seed=seed)
    return pr.u0.astype(np.float32), pr.r.astype(np.float32), pr.beta_l.astype(np.float32), \
        pr.beta_r.astype(np.float32)


def dev(*arrs):
    return [torch.tensor(np.ascontiguousarray(x), device=DEV) for x in arrs]


def rel_rows(got, want):
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


def oracle_params(m) -> np.ndarray:
    return S.round_bf16(torch.tensor(get_params(m))).numpy()


def test_num_params_matches_layout():
    for a in (SMALL, FULL):
        m = make_model(a, 2)
        assert B.ge_sno_num_params(m) == S.num_params(a)
        B.ge_sno_destroy(m)


@pytest.mark.parametrize("a,batch", [(SMALL, 5), (FULL, 3)])
@pytest.mark.parametrize("split,tol", [(1, 1e-4), (0, 3e-2)])
def test_forward_parity(a, batch, split, tol):
    m = make_model(a, 8, split=split)
    u0, r, bl, br = problem_batch(a, batch, 11)
    pred = torch.empty(batch, a.n, dtype=torch.float32, device=DEV)
    B.ge_sno_forward(m, batch, *dev(u0, r, bl, br), pred)
    torch.cuda.synchronize()
    want = S.predict(oracle_params(m), a, u0, r, bl, br)
    err = rel_rows(pred.cpu().numpy().astype(np.float64), want)
    assert np.all(err <= tol), err
    B.ge_sno_destroy(m)


def blocks(a: S.Arch, g: np.ndarray) -> dict:
    return {k: v.numpy() for k, v in S.unpack(torch.tensor(g), a).items()}


@pytest.mark.parametrize("a,batch", [(SMALL, 4), (FULL, 2)])
def test_gradient_parity(a, batch):
    m = make_model(a, 8, split=1)
    u0, r, bl, br = problem_batch(a, batch, 12)
    target = (u0 + 0.1 * np.random.default_rng(13).standard_normal(u0.shape)).astype(np.float32)
    loss = torch.empty(batch, dtype=torch.float32, device=DEV)
    grads = torch.empty(B.ge_sno_num_params(m), dtype=torch.float32, device=DEV)
    B.ge_sno_loss_grad(m, batch, *dev(u0, r, bl, br, target), loss, grads)
    torch.cuda.synchronize()
    want_loss, want_grad = S.loss_and_grad(oracle_params(m), a, u0, r, bl, br, target)
    np.testing.assert_allclose(loss.cpu().numpy(), want_loss, rtol=1e-4)
    got = blocks(a, grads.cpu().numpy().astype(np.float64))
    ref = blocks(a, want_grad)
    for k in ref:
        den = max(np.linalg.norm(ref[k]), 1e-12)
        assert np.linalg.norm(got[k] - ref[k]) <= 2e-3 * den, (k, np.linalg.norm(got[k] - ref[k]) / den)
    B.ge_sno_destroy(m)


def test_adam_step_matches_reference_update():
    a = SMALL
    m = make_model(a, 4, split=1)
    u0, r, bl, br = problem_batch(a, 3, 14)
    target = np.roll(u0, 3, axis=1).astype(np.float32)
    p0 = get_params(m).astype(np.float64)
    B.ge_sno_loss_grad(m, 3, *dev(u0, r, bl, br, target), None, None)
    B.ge_sno_adam_step(m, 1e-3)
    torch.cuda.synchronize()
    p1 = get_params(m).astype(np.float64)
    _, g = S.loss_and_grad(S.round_bf16(torch.tensor(p0)).numpy(), a, u0, r, bl, br, target)
    # first bias-corrected Adam step: p - lr * g / (|g| + eps) (elementwise sign step)
    want = p0 - 1e-3 * g / (np.abs(g) + 1e-8)
    big = np.abs(g) > 1e-4 * np.abs(g).max()
    np.testing.assert_allclose(p1[big], want[big], rtol=0, atol=2e-6)


def test_invalid_arguments_are_rejected():
    m = make_model(SMALL, 4)
    x = torch.zeros(5 * SMALL.n, dtype=torch.float32, device=DEV)
    v = torch.zeros(5, dtype=torch.float32, device=DEV)
    with pytest.raises(B.GeError):
        B.ge_sno_forward(m, 5, x, v, v, v, x)     # batch > max_batch
    with pytest.raises(B.GeError):
        B.ge_sno_set_precision(m, 2)
    with pytest.raises(B.GeError):
        B.ge_sno_adam_step(m, float("nan"))
    B.ge_sno_destroy(m)


@pytest.fixture(scope="module")
def trained():
    """The full-size surrogate trained briefly on GE trajectories (K = 256)."""
    data = SG.make_training_set(1024, K=256, jumps=8, seed=inputs.SEED_BASE + 40)
    held = SG.make_training_set(64, K=256, jumps=8, seed=inputs.SEED_BASE + 41)
    sur = SG.Surrogate(max_batch=64, seed=3)
    untrained = sur.evaluate(held)
    losses = sur.train(data, steps=600, batch=32, lr=2e-3, warmup=50)
    yield sur, data, held, untrained, losses
    sur.close()


def test_training_reduces_the_loss(trained):
    sur, data, held, untrained, losses = trained
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.2 * losses[:20].mean()


def test_trained_network_gains_over_the_baselines(trained):
    """What training buys: one jump of the trained network is far closer to
    GE than the same network untrained and than the do-nothing prediction
    u_K = u_0, on trajectories it has not seen."""
    sur, data, held, untrained, _ = trained
    err = sur.evaluate(held)
    ident = (torch.linalg.vector_norm(held.x - held.y, dim=1) / torch.linalg.vector_norm(held.y, dim=1)).cpu().numpy()
    assert np.median(err) < 0.1 * np.median(untrained)
    assert np.median(err) < 0.5 * np.median(ident)


def ge_reference(u0, r, bl, br, steps, prec=B.GE_F32):
    ref = u0.to(torch.float64 if prec == B.GE_F64 else torch.float32).clone()
    ge = SG.GEBatch(r.double().cpu().numpy(), bl.double().cpu().numpy(), br.double().cpu().numpy(),
                    u0.shape[1], prec)
    ge.run(ref, steps)
    torch.cuda.synchronize()
    ge.close()
    return ref.float()


def test_fallback_takes_over_when_the_sample_misses(trained):
    """A tolerance no network meets: every problem ends up with GE's answer."""
    sur = trained[0]
    pr = inputs.surrogate_problems(300, 1024, seed=inputs.SEED_BASE + 42)
    u0, r, bl, br = dev(pr.u0.astype(np.float32), *(x.astype(np.float32) for x in (pr.r, pr.beta_l, pr.beta_r)))
    out, rep = SG.solve_with_fallback(sur, u0, r, bl, br, jumps=2, tol=1e-9, sample_frac=0.05)
    assert rep.fell_back_all and rep.n_sample_over_tol > 0
    assert torch.equal(out, ge_reference(u0, r, bl, br, 2 * 256))


def test_fallback_replaces_flagged_and_sampled_rows(trained):
    sur = trained[0]
    pr = inputs.surrogate_problems(200, 1024, seed=inputs.SEED_BASE + 43)
    r_np = pr.r.astype(np.float32)
    r_np[[5, 77]] = 6.0                           # outside the trained range: flagged
    u0, r, bl, br = dev(pr.u0.astype(np.float32), r_np, pr.beta_l.astype(np.float32), pr.beta_r.astype(np.float32))
    out, rep = SG.solve_with_fallback(sur, u0, r, bl, br, jumps=1, tol=1e9, sample_frac=0.02)
    assert not rep.fell_back_all and rep.n_flagged == 2
    ref = ge_reference(u0, r, bl, br, 256)
    rows = np.union1d(rep.sample, [5, 77])
    assert torch.equal(out[rows], ref[rows])
    surrogate_only = sur.predict(u0, r, bl, br)
    others = np.setdiff1d(np.arange(200), rows)
    assert torch.equal(out[others], surrogate_only[others])


def test_non_finite_predictions_are_flagged():
    a = SG.SnoArch()
    sur = SG.Surrogate(a, max_batch=16, seed=5)
    p = sur.params()
    p[:] = float("nan")
    sur.set_params(p)
    pr = inputs.surrogate_problems(40, a.n, seed=inputs.SEED_BASE + 44)
    u0, r, bl, br = dev(pr.u0.astype(np.float32), *(x.astype(np.float32) for x in (pr.r, pr.beta_l, pr.beta_r)))
    out, rep = SG.solve_with_fallback(sur, u0, r, bl, br, jumps=1, tol=1e-3)
    assert rep.n_flagged == 40 and not rep.fell_back_all
    assert torch.equal(out, ge_reference(u0, r, bl, br, 256))
    sur.close()


def test_arbiter_row_helpers_match_numpy():
    """The fallback arbiter's row kernels: non-finite flags, gather, scatter
    (indices outside the rows skipped) and the per-row relative L2 error
    (FP64 sums; inf for non-finite rows or a zero reference that differs,
    NaN for an index outside the rows)."""
    a = SMALL
    m = make_model(a, 8, split=1)
    rng = np.random.default_rng(41)
    P = 37
    u = rng.standard_normal((P, a.n)).astype(np.float32)
    u[3, 5] = np.nan
    u[10, 0] = np.inf
    u[36, a.n - 1] = -np.inf
    ud = torch.tensor(u, device=DEV)
    flags = torch.empty(P, dtype=torch.int32, device=DEV)
    B.ge_sno_rows_nonfinite(m, ud, flags)
    assert np.array_equal(flags.cpu().numpy(), (~np.isfinite(u).all(axis=1)).astype(np.int32))

    idx = np.array([0, 7, 36, -1, P, 12, 7], dtype=np.int64)
    idd = torch.tensor(idx, device=DEV)
    dst = torch.full((idx.size, a.n), 5.0, device=DEV)
    B.ge_sno_rows_gather(m, ud, idd, dst)
    got = dst.cpu().numpy()
    for i, k in enumerate(idx):
        want = u[k] if 0 <= k < P else np.full(a.n, 5.0, np.float32)
        assert np.array_equal(got[i], want, equal_nan=True)

    tgt = torch.zeros(P, a.n, device=DEV)
    src = torch.tensor(rng.standard_normal((idx.size, a.n)).astype(np.float32), device=DEV)
    sidx = torch.tensor(np.array([4, 9, -3, 40, 30], dtype=np.int64), device=DEV)
    B.ge_sno_rows_scatter(m, tgt, sidx, src)
    want = np.zeros((P, a.n), np.float32)
    sh = src.cpu().numpy()
    for i, k in enumerate([4, 9, -3, 40, 30]):
        if 0 <= k < P:
            want[k] = sh[i]
    assert np.array_equal(tgt.cpu().numpy(), want)

    ref = rng.standard_normal((idx.size, a.n)).astype(np.float32)
    ref[5] = 0.0
    a_rows = u.copy()
    a_rows[12] = 0.0   # row 12 against the zero reference row 5: error 0
    ad = torch.tensor(a_rows, device=DEV)
    err = torch.empty(idx.size, dtype=torch.float32, device=DEV)
    B.ge_sno_rows_rel_err(m, ad, idd, torch.tensor(ref, device=DEV), err)
    got = err.cpu().numpy()
    for i, k in enumerate(idx):
        if not 0 <= k < P:
            assert np.isnan(got[i])
            continue
        d = a_rows[k].astype(np.float64) - ref[i]
        if not np.all(np.isfinite(d)):
            assert got[i] == np.inf
        elif not np.any(ref[i]):
            assert got[i] == (0.0 if not np.any(d) else np.inf)
        else:
            w = np.linalg.norm(d) / np.linalg.norm(ref[i].astype(np.float64))
            assert abs(got[i] - w) <= 1e-6 * w
    B.ge_sno_destroy(m)


@pytest.mark.parametrize("batch", [1, 3, 600])
def test_tensor_core_path_matches_the_mma_path(batch):
    """Inference on the tcgen05 path (fused layers and projection as
    tensor-core MMAs with TMEM accumulators) computes the same BF16 network
    as the mma.sync path: the network's part of the prediction (pred - u0)
    agrees to 1e-2 relative L2 per problem (only FP32 accumulation order, and
    the BF16 roundings after it, differ), and small batches also match the
    FP64 reference at the BF16 tolerance.  600 problems make 4800 row tiles,
    several per CTA, so both stages and both accumulators are reused."""
    m = make_model(FULL, batch, seed=3, split=0)
    assert B.ge_sno_get_tensor_cores(m) == 1
    u0, r, bl, br = problem_batch(FULL, batch, 17)
    args = dev(u0, r, bl, br)
    p_tc = torch.empty(batch, FULL.n, dtype=torch.float32, device=DEV)
    B.ge_sno_forward(m, batch, *args, p_tc)
    B.ge_sno_sync(m)
    B.ge_sno_set_tensor_cores(m, 0)
    assert B.ge_sno_get_tensor_cores(m) == 0
    p_mma = torch.empty_like(p_tc)
    B.ge_sno_forward(m, batch, *args, p_mma)
    B.ge_sno_sync(m)
    B.ge_sno_set_tensor_cores(m, 1)
    B.ge_sno_set_precision(m, 1)
    assert B.ge_sno_get_tensor_cores(m) == 0   # split mode keeps the mma.sync path
    B.ge_sno_set_precision(m, 0)
    a_tc, a_mma = p_tc.cpu().numpy().astype(np.float64), p_mma.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(a_tc))
    err = rel_rows(a_tc - u0, a_mma - u0)
    assert np.all(err <= 1e-2), err.max()
    if batch <= 3:
        want = S.predict(oracle_params(m), FULL, u0, r, bl, br)
        assert np.all(rel_rows(a_tc, want) <= 3e-2)
    B.ge_sno_destroy(m)


def test_tensor_core_path_follows_parameter_changes():
    """The tcgen05 path keeps the operands it derives from the weights (BF16
    rounding, K-major copies, K-major spectral weights) from one call to the
    next.  After ge_sno_set_params, and after a training step, its output is
    bit-for-bit that of a second model given the same parameters (same
    kernels, same inputs), and differs from the output before the change."""
    batch = 4
    m = make_model(FULL, batch, seed=3, split=0)
    ref = make_model(FULL, batch, seed=9, split=0)
    u0, r, bl, br = problem_batch(FULL, batch, 23)
    args = dev(u0, r, bl, br)

    def run(model):
        out = torch.empty(batch, FULL.n, dtype=torch.float32, device=DEV)
        B.ge_sno_forward(model, batch, *args, out)
        B.ge_sno_sync(model)
        return out.cpu().numpy()

    def same_as_fresh(model):
        p = torch.tensor(get_params(model), device=DEV)
        B.ge_sno_set_params(ref, p)
        return np.array_equal(run(model), run(ref))

    before = run(m)
    assert same_as_fresh(m)
    p = torch.tensor(get_params(m), device=DEV)
    B.ge_sno_set_params(m, p * 0.75)
    after_set = run(m)
    assert not np.array_equal(after_set, before)
    assert same_as_fresh(m)
    target = torch.tensor(u0, device=DEV)
    B.ge_sno_train_step(m, batch, *args, target, 1e-3)
    after_step = run(m)
    assert not np.array_equal(after_step, after_set)
    assert same_as_fresh(m)
    B.ge_sno_destroy(m)
    B.ge_sno_destroy(ref)
