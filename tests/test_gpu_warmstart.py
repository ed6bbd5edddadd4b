"""Learned warm start on the GPU: forward pass, gradients and Adam against the
FP64 oracle (``oracle/warmstart.py``), training, the zero-guess fallback, and
what the trained network gains over the zero initial guess.

BF16 tolerances: the GPU rounds every activation, the aggregated features, the
backpropagated dz and the weights to BF16 (relative rounding 2^-9), over four
layers; per-tensor relative errors of 2e-2 with cosine similarity >= 0.999 are
the bar, the loss within 1e-2.
"""
import numpy as np
import pytest

import gl_inputs as gi
from oracle import warmstart as ows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
INV_SQRT3 = 1.0 / np.sqrt(3.0)
# (dim, N, mu, field): n = 2025 and 2197 nodes = 16 and 18 tiles of 128 with ragged tails
CASES = [(2, 45, 1.0, (0.0, 0.0, 1.0)), (3, 13, 1.0, (INV_SQRT3, INV_SQRT3, INV_SQRT3))]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cosine(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim,N,mu,field", CASES)
def test_forward_matches_oracle(oracle_mod, dim, N, mu, field):
    om = oracle_mod.Mesh(dim, N, mu, field)
    g = ows.Graph(om)
    psi = gi.disk(om.n, 21)
    b = gi.complex_normal(om.n, 22)
    theta = gi.warmstart_init(3)
    m = gl.gl_mesh_create(dim, N, mu, field)
    ws = gl.gl_warmstart_create(theta)
    try:
        x0 = torch.zeros(om.n, dtype=torch.complex128, device=DEV)
        gl.gl_warmstart_predict(ws, m, dev(psi), dev(b), x0)
        torch.cuda.synchronize()
        expect = ows.predict(theta.astype(np.float64), g, psi, b)
        got = x0.cpu().numpy()
        assert rel(got, expect) <= 2e-2, rel(got, expect)
        # scale equivariance holds exactly up to the FP64 scaling of the output
        x1 = torch.zeros_like(x0)
        gl.gl_warmstart_predict(ws, m, dev(psi), dev(4.0 * b), x1)
        np.testing.assert_allclose(x1.cpu().numpy(), 4.0 * got, rtol=1e-6, atol=1e-6 * np.abs(got).max())
    finally:
        gl.gl_warmstart_destroy(ws)
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("dim,N,mu,field", CASES)
def test_gradient_matches_oracle(oracle_mod, dim, N, mu, field):
    om = oracle_mod.Mesh(dim, N, mu, field)
    g = ows.Graph(om)
    psi = gi.disk(om.n, 31)
    b = gi.complex_normal(om.n, 32)
    theta = gi.warmstart_init(4)
    m = gl.gl_mesh_create(dim, N, mu, field)
    ws = gl.gl_warmstart_create(theta)
    try:
        L, grad = gl.gl_warmstart_grad(ws, m, dev(psi), dev(b))
        Lo, go = ows.loss_and_grad(theta.astype(np.float64), g, psi, b)
        assert abs(L - Lo) <= 1e-2 * Lo, (L, Lo)
        Ws, U = ows.split(np.arange(ows.NPARAM))
        for name, idx in [("W0", Ws[0]), ("W1", Ws[1]), ("W2", Ws[2]), ("W3", Ws[3]), ("U", U)]:
            a, e = grad[idx.ravel()].astype(np.float64), go[idx.ravel()]
            assert rel(a, e) <= 2e-2 and cosine(a, e) >= 0.999, (name, rel(a, e), cosine(a, e))
            assert np.all(grad[Ws[0][ows.C - 1]] == 0.0)
    finally:
        gl.gl_warmstart_destroy(ws)
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("dim,N,mu,field", CASES)
def test_hint_forward_and_gradient_match_oracle(oracle_mod, dim, N, mu, field):
    """With a hint: the FP64 minimal-residual multiple alpha a matches the oracle's
    to FP64 rounding (zero network), the network's correction at the BF16 bar,
    and the gradient (including the weights reading the hint channels) too."""
    om = oracle_mod.Mesh(dim, N, mu, field)
    g = ows.Graph(om)
    psi = gi.disk(om.n, 41)
    b = gi.complex_normal(om.n, 42)
    a = gi.complex_normal(om.n, 43) + 0.5 * b
    m = gl.gl_mesh_create(dim, N, mu, field)
    ws = gl.gl_warmstart_create(np.zeros(gl.GL_WS_NPARAM, np.float32))
    try:
        x0 = torch.zeros(om.n, dtype=torch.complex128, device=DEV)
        gl.gl_warmstart_predict(ws, m, dev(psi), dev(b), x0, hint=dev(a))
        torch.cuda.synchronize()
        base = ows.predict(np.zeros(ows.NPARAM), g, psi, b, a)
        assert rel(x0.cpu().numpy(), base) <= 1e-12
        theta = gi.warmstart_init(8)
        gl.gl_warmstart_set_params(ws, theta)
        gl.gl_warmstart_predict(ws, m, dev(psi), dev(b), x0, hint=dev(a))
        torch.cuda.synchronize()
        expect = ows.predict(theta.astype(np.float64), g, psi, b, a)
        got = x0.cpu().numpy()
        assert rel(got - base, expect - base) <= 2e-2, rel(got - base, expect - base)
        L, grad = gl.gl_warmstart_grad(ws, m, dev(psi), dev(b), hint=dev(a))
        Lo, go = ows.loss_and_grad(theta.astype(np.float64), g, psi, b, a)
        assert abs(L - Lo) <= 1e-2 * Lo, (L, Lo)
        Ws, U = ows.split(np.arange(ows.NPARAM))
        for name, idx in [("W0", Ws[0]), ("W3", Ws[3]), ("U", U),
                          ("W0 hint columns", np.concatenate([Ws[0][:, 6], Ws[0][:, 7], Ws[0][:, ows.C + 6],
                                                              Ws[0][:, ows.C + 7]]))]:
            x, e = grad[idx.ravel()].astype(np.float64), go[idx.ravel()]
            # two more BF16-rounded input channels (the hint pair) than without a
            # hint: 3e-2 per tensor (measured 2.1-2.9e-2), cosine >= 0.999
            assert rel(x, e) <= 3e-2 and cosine(x, e) >= 0.999, (name, rel(x, e), cosine(x, e))
    finally:
        gl.gl_warmstart_destroy(ws)
        gl.gl_mesh_destroy(m)


def test_adam_matches_oracle():
    theta = gi.warmstart_init(5)
    ws = gl.gl_warmstart_create(theta)
    try:
        th = theta.astype(np.float64)
        mm = np.zeros_like(th)
        vv = np.zeros_like(th)
        rng = gi.rng(8)
        for t in range(1, 4):
            grad = (rng.standard_normal(th.size) * 1e-2).astype(np.float32)
            gl.gl_warmstart_adam_step(ws, grad, 1e-3)
            th, mm, vv = ows.adam_step(th, grad.astype(np.float64), mm, vv, t, 1e-3)
        np.testing.assert_allclose(gl.gl_warmstart_get_params(ws), th, rtol=1e-5, atol=1e-7)
    finally:
        gl.gl_warmstart_destroy(ws)


def true_relres(om, psi, b, x):
    vol = om.volumes()
    r = b - om.jacobian(psi, x)
    return np.sqrt(np.sum(vol * np.abs(r) ** 2) / np.sum(vol * np.abs(b) ** 2))


def test_training_fallback_and_solve(oracle_mod):
    """Train on 8 right-hand sides, solve a ninth from the network's guess; a
    zero network and a wildly scaled one must both fall back to x0 = 0."""
    N, mu = 64, 1.0
    om = oracle_mod.Mesh(2, N, mu)
    n = om.n
    psi = gi.disk(n, 1)
    m = gl.gl_mesh_create(2, N, mu)
    ws = gl.gl_warmstart_create(gi.warmstart_init(6))
    try:
        psis = [dev(psi)] * 8
        bs = [dev(gi.complex_normal(n, 300 + j)) for j in range(8)]
        losses = gl.gl_warmstart_train(ws, [m] * 8, psis, bs, steps=300, batch=2, lr=2e-3)
        first, last = float(np.mean(losses[:10])), float(np.mean(losses[-10:]))
        print(f"training loss {first:.3f} -> {last:.3f}")
        assert np.all(np.isfinite(losses))
        assert last < 0.5 * first and last < 0.5
        b = gi.complex_normal(n, 1)
        opts = gl.options(max_coarse=64)
        x = torch.zeros(n, dtype=torch.complex128, device=DEV)
        st0, inf0 = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x, opts)
        assert st0 == 0 and inf0.warmstart_used == 0
        x0 = torch.zeros_like(x)
        gl.gl_warmstart_predict(ws, m, dev(psi), dev(b), x0)
        r0 = true_relres(om, psi, b, x0.cpu().numpy())
        assert r0 < 1.0
        opts.warmstart = ws.value
        x.fill_(123.0)  # ignored: the network supplies the initial guess
        st1, inf1 = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x, opts)
        print(f"guess residual {r0:.3f}; iterations {inf0.iters} (zero guess) vs {inf1.iters} (warm start)")
        assert st1 == 0 and inf1.warmstart_used == 1
        assert true_relres(om, psi, b, x.cpu().numpy()) <= 1.01e-10
        assert inf1.iters <= inf0.iters + 1
        # fallbacks: the zero network gives x0 = 0 (not better than zero)...
        gl.gl_warmstart_set_params(ws, np.zeros(gl.GL_WS_NPARAM, np.float32))
        x.zero_()
        st2, inf2 = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x, opts)
        assert st2 == 0 and inf2.warmstart_used == 0 and inf2.iters == inf0.iters
        # ... and a network whose guess is far too large is rejected
        big = gi.warmstart_init(6) * 40.0
        gl.gl_warmstart_set_params(ws, big)
        st3, inf3 = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x, opts)
        assert st3 == 0 and inf3.warmstart_used == 0 and inf3.iters == inf0.iters
        assert true_relres(om, psi, b, x.cpu().numpy()) <= 1.01e-10
    finally:
        gl.gl_warmstart_destroy(ws)
        gl.gl_mesh_destroy(m)


def test_continuation_gain(oracle_mod):
    """Natural-parameter continuation in mu on a 2D square (from psi = 1 at mu = 0,
    Sec. 4): Newton steps J d = -GL(psi), psi += d, until ||GL(psi)||_R <= 1e-8
    (below that the round-off in GL(psi) has a component along the near-null
    direction i psi of J that no solve can reduce 1e-10-fold).  Every Newton
    system comes with a hint: the correction of the same Newton step at the
    previous mu.  The network is trained on the systems of the first half of the
    continuation and used on the second half; every warm-started solve is
    compared with the zero-guess solve of the same system and with the guess the
    hint alone gives (its minimal-residual multiple; the solve then runs no
    network, and the multiple equals the zero network's guess).  Reported:
    the guesses' relative residuals and the iterations and time they save."""
    N, steps = 64, 24
    mus = [2.0 * (s + 1) / steps for s in range(steps)]
    n = N * N
    psi = torch.ones(n, dtype=torch.complex128, device=DEV)
    opts = gl.options(max_coarse=64)
    train = dict(m=[], psi=[], b=[], hint=[])
    held = []
    meshes = []
    prev = []  # the Newton corrections at the previous mu
    try:
        for s, mu in enumerate(mus):
            m = gl.gl_mesh_create(2, N, mu)
            meshes.append(m)
            cur = []
            for it in range(8):
                r = torch.zeros_like(psi)
                gl.gl_residual(m, psi, r)
                # sqrt(sum h^2 |r|^2) >= ||r||_R since every |V_i| <= h^2
                gnorm = float(torch.sqrt(torch.sum(torch.abs(r) ** 2))) / (N - 1)
                if gnorm <= 1e-8:
                    break
                b = -r
                d = torch.zeros_like(psi)
                st, inf = gl.gl_jacobian_solve(m, psi, None, b, d, opts)
                assert st == 0
                hint = prev[it] if it < len(prev) else None
                if hint is not None:
                    if s < steps // 2:
                        train["m"].append(m)
                        train["psi"].append(psi.clone())
                        train["b"].append(b.clone())
                        train["hint"].append(hint)
                    else:
                        held.append((m, mu, psi.clone(), b.clone(), hint, inf.iters, inf.solve_ms))
                cur.append(d.clone())
                psi = psi + d
            prev = cur
        assert len(train["b"]) >= 8 and len(held) >= 8
        ws = gl.gl_warmstart_create(gi.warmstart_init(12))
        try:
            losses = gl.gl_warmstart_train(ws, train["m"], train["psi"], train["b"], steps=400, batch=4, lr=2e-3,
                                           hints=train["hint"])
            assert losses[-20:].mean() < losses[:20].mean()
            trained = gl.gl_warmstart_get_params(ws)
            out = {}
            for label, params in (("hint alone", np.zeros(gl.GL_WS_NPARAM, np.float32)), ("hint + network", trained)):
                gl.gl_warmstart_set_params(ws, params)
                its = used = 0
                ms = 0.0
                res = []
                for m, mu, p, b, hint, iters0, ms0 in held:
                    x0 = torch.zeros_like(b)
                    gl.gl_warmstart_predict(ws, m, p, b, x0, hint=hint)
                    om = oracle_mod.Mesh(2, N, mu)
                    pn, bn = p.cpu().numpy(), b.cpu().numpy()
                    res.append(true_relres(om, pn, bn, x0.cpu().numpy()))
                    wopts = gl.options(max_coarse=64)
                    if label != "hint alone":
                        wopts.warmstart = ws.value
                    wopts.warmstart_hint = hint.data_ptr()
                    x = torch.zeros_like(b)
                    st, inf = gl.gl_jacobian_solve(m, p, None, b, x, wopts)
                    assert st == 0 and true_relres(om, pn, bn, x.cpu().numpy()) <= 1.01e-10
                    assert inf.iters <= iters0 + 1
                    its += inf.iters
                    used += inf.warmstart_used
                    ms += inf.solve_ms
                out[label] = (its, used, ms, res)
            it0 = sum(h[5] for h in held)
            ms0 = sum(h[6] for h in held)
            print(f"continuation: {len(train['b'])} training solves, {len(held)} held-out solves, zero guess "
                  f"{it0} iterations ({ms0:.1f} ms)")
            for label, (its, used, ms, res) in out.items():
                print(f"  {label}: guess residual median {np.median(res):.2e} (max {max(res):.2e}); used "
                      f"{used}/{len(held)}; iterations {it0} -> {its}; solve ms {ms0:.1f} -> {ms:.1f}")
            # both guesses save iterations over the zero guess (the method without a
            # warm start); the network lowers the guess's residual below the hint's
            # multiple's but, measured, saves no further iterations
            assert out["hint alone"][0] < it0 and out["hint + network"][0] < it0
            assert np.median(out["hint + network"][3]) < np.median(out["hint alone"][3])
        finally:
            gl.gl_warmstart_destroy(ws)
    finally:
        for m in meshes:
            gl.gl_mesh_destroy(m)
