"""The differentiable form: dA = dC B^T and dB = A^T dC through the cascade
(C ABI ddgemm_backward and the torch.autograd.Function), for the loss
L = sum(W * C) with W an FP64x2 matrix, so dC = W.

Checks: the oracle's own double-double products W B^T and A^T W (within the
1e-28 |.||.| contract for uniform entries and the paper's bound otherwise),
all four transposition cases, central double-double finite differences of
L at 64^3 (L is linear in A and B, so the difference quotient is exact up
to the FP64x2 rounding of L), and the 2048^3 workload on sampled entries."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dd  # noqa: E402
from tests import exact  # noqa: E402
from tests.bounds import paper_bound  # noqa: E402
from workloads import dd_matrix, gemm_inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CONTRACT = 1e-28


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04353_gb300 import autograd, ops
    return ops, autograd


def dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def host(*tensors):
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in tensors]


def close(got_hi, got_lo, want_hi, want_lo, x_hi, y_hi, contract):
    diff = np.abs((got_hi - want_hi) + (got_lo - want_lo))
    absxy = np.abs(x_hi) @ np.abs(y_hi)
    k = x_hi.shape[1]
    assert np.all(diff <= paper_bound(x_hi, y_hi) + 4 * (k + 2) * 2.0 ** -106 * absxy)
    if contract:
        assert np.all(diff <= CONTRACT * absxy)


@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_backward_matches_oracle(mods, kind):
    ops, autograd = mods
    m, n, k = 96, 80, 300
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=31)
    w_hi, w_lo = dd_matrix(np.random.default_rng(32), (m, n))
    t = dev(a_hi, a_lo, b_hi, b_lo)
    for x in t:
        x.requires_grad_(True)
    c_hi, c_lo = autograd.ddmatmul(*t)
    torch.autograd.backward((c_hi, c_lo), tuple(dev(w_hi, w_lo)))
    da_hi, da_lo, db_hi, db_lo = host(t[0].grad, t[1].grad, t[2].grad, t[3].grad)
    o_hi, o_lo = dd.ddgemm(w_hi, w_lo, b_hi.T, b_lo.T)          # W B^T
    close(da_hi, da_lo, o_hi, o_lo, w_hi, b_hi.T, kind == "uniform")
    o_hi, o_lo = dd.ddgemm(a_hi.T, a_lo.T, w_hi, w_lo)          # A^T W
    close(db_hi, db_lo, o_hi, o_lo, a_hi.T, w_hi, kind == "uniform")
    # forward output too
    f_hi, f_lo = host(c_hi.detach(), c_lo.detach())
    o_hi, o_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
    close(f_hi, f_lo, o_hi, o_lo, a_hi, b_hi, kind == "uniform")


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_backward_transposed_storage(mods, ta, tb):
    ops, _ = mods
    m, n, k = 70, 50, 260
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, seed=33)
    w_hi, w_lo = dd_matrix(np.random.default_rng(34), (m, n))
    sa = (a_hi.T, a_lo.T) if ta else (a_hi, a_lo)
    sb = (b_hi.T, b_lo.T) if tb else (b_hi, b_lo)
    da_hi, da_lo, db_hi, db_lo = host(*ops.ddgemm_backward(*dev(*sa), *dev(*sb),
                                                          *dev(w_hi, w_lo),
                                                          trans_a=ta, trans_b=tb))
    o_hi, o_lo = dd.ddgemm(w_hi, w_lo, b_hi.T, b_lo.T)
    if ta:
        da_hi, da_lo = da_hi.T, da_lo.T
    close(da_hi, da_lo, o_hi, o_lo, w_hi, b_hi.T, True)
    o_hi, o_lo = dd.ddgemm(a_hi.T, a_lo.T, w_hi, w_lo)
    if tb:
        db_hi, db_lo = db_hi.T, db_lo.T
    close(db_hi, db_lo, o_hi, o_lo, a_hi.T, w_hi, True)


def _loss_row_change(a_hi, a_lo, b_hi, b_lo, w_hi, w_lo, i, l, h):
    """L(A + h e_il) - L(A - h e_il) from row i of C only, with the
    double-double oracle for C and exact rationals for sum(W * C)."""
    out = []
    for sgn in (1.0, -1.0):
        ph, pl = a_hi[i:i + 1].copy(), a_lo[i:i + 1].copy()
        s, e = dd.two_sum(float(ph[0, l]), sgn * h)       # exact perturbation
        ph[0, l], pl[0, l] = s, e + pl[0, l]
        c_hi, c_lo = dd.ddgemm(ph, pl, b_hi, b_lo)
        out.append(sum(exact.dd_fixed(wh, wl) * exact.dd_fixed(ch, cl) for wh, wl, ch, cl in
                       zip(w_hi[i], w_lo[i], c_hi[0], c_lo[0])))
    return out[0] - out[1]                                  # scaled by 2^2148


def test_backward_double_double_finite_differences(mods):
    ops, _ = mods
    m = n = k = 64
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, seed=35)
    w_hi, w_lo = dd_matrix(np.random.default_rng(36), (m, n))
    da_hi, da_lo, db_hi, db_lo = host(*ops.ddgemm_backward(*dev(a_hi, a_lo, b_hi, b_lo),
                                                          *dev(w_hi, w_lo)))
    h = 2.0 ** -20
    rng = np.random.default_rng(37)
    for i, l in zip(rng.integers(0, m, 6), rng.integers(0, k, 6)):
        dl = _loss_row_change(a_hi, a_lo, b_hi, b_lo, w_hi, w_lo, i, l, h)
        fd = float(exact.Fraction(dl, 1 << (2 * exact.SHIFT))) / (2 * h)
        got = da_hi[i, l] + da_lo[i, l]
        scale = float(np.abs(w_hi[i]) @ np.abs(b_hi[l]))
        # the quotient inherits the FP64x2 rounding of L (~2^-100 |L|) / 2h
        assert abs(fd - got) <= 2.0 ** -60 * scale + 2.0 ** -52 * abs(got)
    # dB by the same route, with B perturbed: L is symmetric in the roles
    at_hi, at_lo = np.ascontiguousarray(b_hi.T), np.ascontiguousarray(b_lo.T)
    for l, j in zip(rng.integers(0, k, 4), rng.integers(0, n, 4)):
        # L = sum(W * (A B)) = sum(W^T * (B^T A^T)): perturb row j of B^T
        dl = _loss_row_change(at_hi, at_lo, a_hi.T.copy(), a_lo.T.copy(),
                              np.ascontiguousarray(w_hi.T), np.ascontiguousarray(w_lo.T),
                              j, l, h)
        fd = float(exact.Fraction(dl, 1 << (2 * exact.SHIFT))) / (2 * h)
        got = db_hi[l, j] + db_lo[l, j]
        scale = float(np.abs(a_hi[:, l]) @ np.abs(w_hi[:, j]))
        assert abs(fd - got) <= 2.0 ** -60 * scale + 2.0 ** -52 * abs(got)


def test_backward_2048_sampled(mods):
    """The 2048^3 differentiable workload (entries as the uniform case);
    sampled entries of dA and dB against the double-double oracle."""
    ops, autograd = mods
    n = 2048
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(n, n, n, kind="uniform", seed=0)
    w_hi, w_lo = dd_matrix(np.random.default_rng(1), (n, n))
    t = dev(a_hi, a_lo, b_hi, b_lo)
    for x in t:
        x.requires_grad_(True)
    c_hi, c_lo = autograd.ddmatmul(*t)
    torch.autograd.backward((c_hi, c_lo), tuple(dev(w_hi, w_lo)))
    da_hi, da_lo, db_hi, db_lo = host(t[0].grad, t[1].grad, t[2].grad, t[3].grad)
    rng = np.random.default_rng(2)
    r, c = rng.integers(0, n, 64), rng.integers(0, n, 64)
    bt_hi, bt_lo = np.ascontiguousarray(b_hi.T), np.ascontiguousarray(b_lo.T)
    oh, ol = dd.ddgemm_entries(w_hi, w_lo, bt_hi, bt_lo, r, c)
    absxy = np.array([np.abs(w_hi[i]) @ np.abs(bt_hi[:, j]) for i, j in zip(r, c)])
    assert np.all(np.abs((da_hi[r, c] - oh) + (da_lo[r, c] - ol)) <= CONTRACT * absxy)
    at_hi, at_lo = np.ascontiguousarray(a_hi.T), np.ascontiguousarray(a_lo.T)
    oh, ol = dd.ddgemm_entries(at_hi, at_lo, w_hi, w_lo, r, c)
    absxy = np.array([np.abs(at_hi[i]) @ np.abs(w_hi[:, j]) for i, j in zip(r, c)])
    assert np.all(np.abs((db_hi[r, c] - oh) + (db_lo[r, c] - ol)) <= CONTRACT * absxy)


@pytest.mark.parametrize("variant", [1, 4])
def test_backward_int8_forms_equal_their_forward_products(mods, variant):
    """The backward of the INT8 forms is two products of the same form:
    dA = dC B^T and dB = A^T dC, bit for bit, and close to the oracle."""
    ops, ag = mods
    m, n, k = 150, 40, 300
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, seed=41)
    w_hi, w_lo = dd_matrix(np.random.default_rng(42), (m, n))
    t = dev(a_hi, a_lo, b_hi, b_lo, w_hi, w_lo)
    da_hi, da_lo, db_hi, db_lo = host(*ops.ddgemm_backward(*t, variant=variant))
    fa = host(*ops.ddgemm(t[4], t[5], t[2].T.contiguous(), t[3].T.contiguous(), variant=variant))
    fb = host(*ops.ddgemm(t[0].T.contiguous(), t[1].T.contiguous(), t[4], t[5], variant=variant))
    assert np.array_equal(da_hi, fa[0]) and np.array_equal(da_lo, fa[1])
    assert np.array_equal(db_hi, fb[0]) and np.array_equal(db_lo, fb[1])
    o_hi, o_lo = dd.ddgemm(w_hi, w_lo, b_hi.T, b_lo.T)
    close(da_hi, da_lo, o_hi, o_lo, w_hi, b_hi.T, True)
    # through autograd
    ta = [x.clone().requires_grad_(True) for x in t[:4]]
    c_hi, c_lo = ag.ddmatmul(*ta, variant=variant)
    torch.autograd.backward((c_hi, c_lo), (t[4], t[5]))
    assert np.array_equal(ta[0].grad.cpu().numpy(), da_hi)
    assert np.array_equal(ta[3].grad.cpu().numpy(), db_lo)
