"""The learned proposal on the GPU against the FP64 oracle.

BF16 operands (weights, standardised inputs, hidden activations) with FP32
accumulation against an FP64 network with the same BF16-rounded weights:
outputs within 3e-2 of their spread, gradients within 5e-2 relative norm per
parameter block. Training rows captured from a plain run must equal the
oracle's recomputation (propagation, Philox noise, features). The gain test
runs the method with and without the trained network at the same small L.
"""
import numpy as np
import pytest

from paper_2312_08684_gb300 import Estimator, _binding as abi, workloads as W

pytestmark = pytest.mark.gpu
H, INP, OUTP = 256, 32, 16


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()
    return torch


def bf16(x):
    x = np.ascontiguousarray(x, np.float32)
    b = x.view(np.uint32)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def unpack(theta, n_in, n_out):
    """Padded GPU layout -> the oracle's packed [W1, b1, W2, b2, W3, b3] (BF16 weights, FP32 biases)."""
    o = 0
    W1 = theta[o:o + H * INP].reshape(H, INP); o += H * INP
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + OUTP * H].reshape(OUTP, H); o += OUTP * H
    b3 = theta[o:o + OUTP]
    return np.concatenate([bf16(W1[:, :n_in]).ravel(), b1, bf16(W2).ravel(), b2,
                           bf16(W3[:n_out]).ravel(), b3[:n_out]]).astype(np.float64)


def _prop(torch, kind, params, seed=3):
    p = abi.smap_proposal_create(kind, params, seed=seed)
    n_in, n_out, hid, npar = abi.smap_proposal_dims(p)
    assert hid == H
    return p, n_in, n_out


def test_forward_matches_oracle(oracle, torch):
    p, n_in, n_out = _prop(torch, 4, W.arm_params())
    try:
        rng = np.random.default_rng(1)
        theta, norm = abi.smap_proposal_get_weights(p)
        norm[:n_in] = rng.normal(0, 1, n_in)
        norm[INP:INP + n_in] = rng.uniform(0.5, 2.0, n_in)
        norm[2 * INP:2 * INP + n_out] = rng.normal(0, 0.1, n_out)
        norm[2 * INP + OUTP:2 * INP + OUTP + n_out] = rng.uniform(0.01, 0.1, n_out)
        abi.smap_proposal_set_weights(p, theta, norm)
        feat = np.zeros((300, INP), np.float32)
        feat[:, :n_in] = rng.normal(0, 2, (300, n_in))
        disp = torch.empty((300, n_out), dtype=torch.float32, device="cuda")
        abi.smap_proposal_forward(p, torch.from_numpy(feat).cuda(), disp)
        xn = bf16((feat[:, :n_in] - norm[:n_in]) / norm[INP:INP + n_in])
        o = oracle.mlp_forward(n_in, H, n_out, unpack(theta, n_in, n_out), xn)
        ref = o * norm[2 * INP + OUTP:2 * INP + OUTP + n_out] + norm[2 * INP:2 * INP + n_out]
        got = disp.cpu().numpy()
        spread = np.std(ref, axis=0).max()
        assert np.max(np.abs(got - ref)) <= 3e-2 * spread
    finally:
        abi.smap_proposal_destroy(p)


def test_forward_many_tiles_matches_oracle(oracle, torch):
    """More 128-row tiles than SMs (several per persistent CTA) plus a ragged
    tail: sampled rows against the oracle, the rest must be finite."""
    p, n_in, n_out = _prop(torch, 3, W.clutter_params(), seed=4)
    try:
        rng = np.random.default_rng(5)
        theta, norm = abi.smap_proposal_get_weights(p)
        norm[:n_in] = rng.normal(0, 1, n_in)
        norm[INP:INP + n_in] = rng.uniform(0.5, 2.0, n_in)
        norm[2 * INP:2 * INP + n_out] = rng.normal(0, 0.1, n_out)
        norm[2 * INP + OUTP:2 * INP + OUTP + n_out] = rng.uniform(0.01, 0.1, n_out)
        abi.smap_proposal_set_weights(p, theta, norm)
        R = 152 * 128 * 3 + 77
        feat = np.zeros((R, INP), np.float32)
        feat[:, :n_in] = rng.normal(0, 2, (R, n_in))
        disp = torch.full((R, n_out), float("nan"), dtype=torch.float32, device="cuda")
        abi.smap_proposal_forward(p, torch.from_numpy(feat).cuda(), disp)
        got = disp.cpu().numpy()
        assert np.all(np.isfinite(got))
        rows = np.r_[np.arange(0, R, 41), np.arange(R - 130, R)]
        xn = bf16((feat[rows, :n_in] - norm[:n_in]) / norm[INP:INP + n_in])
        o = oracle.mlp_forward(n_in, H, n_out, unpack(theta, n_in, n_out), xn)
        ref = o * norm[2 * INP + OUTP:2 * INP + OUTP + n_out] + norm[2 * INP:2 * INP + n_out]
        spread = np.std(ref, axis=0).max()
        assert np.max(np.abs(got[rows] - ref)) <= 3e-2 * spread
    finally:
        abi.smap_proposal_destroy(p)


def test_gradient_matches_oracle(oracle, torch):
    p, n_in, n_out = _prop(torch, 3, W.clutter_params())
    try:
        rng = np.random.default_rng(2)
        R = 512
        feat = np.zeros((R, INP), np.float32); feat[:, :n_in] = rng.normal(0, 1, (R, n_in))
        targ = np.zeros((R, OUTP), np.float32); targ[:, :n_out] = rng.normal(0, 1, (R, n_out))
        theta, norm = abi.smap_proposal_get_weights(p)     # identity normalisation
        loss, g = abi.smap_proposal_loss_grad(p, torch.from_numpy(feat).cuda(), torch.from_numpy(targ).cuda())
        Wp = unpack(theta, n_in, n_out)
        lo, G = oracle.mlp_loss_grad(n_in, H, n_out, Wp, bf16(feat[:, :n_in]), targ[:, :n_out])
        assert loss == pytest.approx(lo, rel=2e-2)
        gp = np.concatenate([g[:H * INP].reshape(H, INP)[:, :n_in].ravel(), g[H * INP:H * INP + H],
                             g[H * INP + H:H * INP + H + H * H], g[H * INP + H + H * H:H * INP + 2 * H + H * H],
                             g[H * INP + 2 * H + H * H:H * INP + 2 * H + H * H + OUTP * H].reshape(OUTP, H)[:n_out].ravel(),
                             g[-OUTP:][:n_out]])
        sizes = [H * n_in, H, H * H, H, n_out * H, n_out]
        o = 0
        for k, s in enumerate(sizes):
            a, b = gp[o:o + s], G[o:o + s]
            assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b), f"block {k}"
            o += s
        # padding stays untouched: zero gradient on the unused inputs / outputs
        assert np.all(g[:H * INP].reshape(H, INP)[:, n_in:] == 0)
    finally:
        abi.smap_proposal_destroy(p)


def test_training_fits_a_teacher(torch):
    p, n_in, n_out = _prop(torch, 4, W.arm_params(), seed=5)
    q, _, _ = _prop(torch, 4, W.arm_params(), seed=77)
    try:
        rng = np.random.default_rng(3)
        R = 1 << 16
        feat = np.zeros((R, INP), np.float32); feat[:, :n_in] = rng.normal(0, 1, (R, n_in))
        fd = torch.from_numpy(feat).cuda()
        disp = torch.empty((R, n_out), dtype=torch.float32, device="cuda")
        abi.smap_proposal_forward(q, fd, disp)             # the teacher
        targ = torch.zeros((R, OUTP), dtype=torch.float32, device="cuda")
        targ[:, :n_out] = disp
        abi.smap_proposal_fit_normalization(p, fd, targ)
        curve = abi.smap_proposal_train(p, fd, targ, 600, 2048, 2e-3, 2e-4)
        assert np.all(np.isfinite(curve))
        assert np.mean(curve[-20:]) < 0.1 * np.mean(curve[:5])
    finally:
        abi.smap_proposal_destroy(p)
        abi.smap_proposal_destroy(q)


def test_capture_rows_match_oracle(oracle, torch):
    wl = W.make_planar_arm(B=2, T=4, N=16, L=5)
    p, n_in, n_out = _prop(torch, wl.kind, wl.params)
    try:
        with Estimator.from_workload(wl) as est:
            est.run_batch(wl.y)
            hist = est.history()
            rows_max = wl.B * wl.maxT * wl.N
            feat = torch.empty((rows_max, INP), dtype=torch.float32, device="cuda")
            targ = torch.empty((rows_max, OUTP), dtype=torch.float32, device="cuda")
            n = abi.smap_proposal_capture(p, est.h, feat, targ)
        assert n == rows_max
        feat, targ = feat.cpu().numpy(), targ.cpu().numpy()
        m = oracle.Model(wl.kind, wl.params)
        r = 0
        for b in range(wl.B):
            for t in range(1, wl.maxT + 1):
                for i in range(wl.N):
                    prev = wl.x0[b] if t == 1 else hist[b, t - 2, i].astype(np.float64)
                    u = m.transition(t, prev) + np.sqrt(m.q) * oracle.normals(wl.seed, b, t, i, wl.d)
                    f = oracle.proposal_features(wl.kind, wl.params, u, wl.y[b, t - 1].astype(np.float64))
                    ns = wl.d // 2          # the arm's score block: the 7 angles
                    k = len(f) - ns
                    assert np.allclose(feat[r, :k], f[:k], rtol=1e-5, atol=2e-5)
                    # the score amplifies FP32 kinematics (fast sincos) by 1/r = 1e4
                    assert np.allclose(feat[r, k:len(f)], f[k:], rtol=1e-3, atol=1e-4 * max(1.0, np.abs(f[k:]).max()))
                    assert np.all(feat[r, len(f):] == 0)
                    assert np.allclose(targ[r, :wl.d], hist[b, t - 1, i] - u, rtol=1e-4, atol=2e-6)
                    r += 1
    finally:
        abi.smap_proposal_destroy(p)


def test_untrained_proposal_stays_finite(torch):
    """Random weights and identity scaling give wild displacements; the
    clamp at 8 standard deviations keeps the method finite."""
    wl = W.make_clutter_cv(B=6, Tmin=12, Tmax=12, N=64, L=3)
    p, _, _ = _prop(torch, wl.kind, wl.params, seed=21)
    try:
        assert np.isfinite(_mean_J(wl, 3, p))
    finally:
        abi.smap_proposal_destroy(p)


def _mean_J(wl, L, prop=None):
    with Estimator.from_workload(wl, L=L) as est:
        if prop is not None:
            abi.smap_set_proposal(est.h, prop, L)
        path, J = est.run_batch(wl.y, wl.T, wl.Nseq)
        steps = np.empty(wl.B, np.int32)
        abi.smap_get_steps(est.h, steps)
    # every sequence ran all its steps and ended with a finite score
    assert np.array_equal(steps, wl.T)
    assert np.all(np.isfinite(J))
    assert np.all(np.isfinite(path[np.arange(wl.B), wl.T]))
    return float(np.mean(J))


@pytest.mark.parametrize("which", ["arm", "clutter"])
def test_learned_proposal_gains_over_plain_at_equal_iterations(torch, which):
    """Train on plain L=50 runs, then compare the MAP log-posterior of the
    learned initialisation + L=5 against plain L=5 (and plain L=50) on fresh
    sequences: the network must close part of the gap."""
    mk = {"arm": lambda B, s: W.make_planar_arm(B=B, T=30, N=256, L=50, seed=s),
          "clutter": lambda B, s: W.make_clutter_cv(B=B, Tmin=30, Tmax=30, N=256, L=50, seed=s)}[which]
    train_wl = mk(48, 11)
    p, n_in, n_out = _prop(torch, train_wl.kind, train_wl.params, seed=9)
    try:
        rows = train_wl.B * train_wl.maxT * train_wl.N
        feat = torch.empty((rows, INP), dtype=torch.float32, device="cuda")
        targ = torch.empty((rows, OUTP), dtype=torch.float32, device="cuda")
        with Estimator.from_workload(train_wl) as est:
            est.run_batch(train_wl.y, train_wl.T, train_wl.Nseq)
            n = abi.smap_proposal_capture(p, est.h, feat, targ)
        abi.smap_proposal_fit_normalization(p, feat[:n], targ[:n])
        curve = abi.smap_proposal_train(p, feat[:n], targ[:n], 1500, 4096, 1e-3, 1e-4)
        assert np.mean(curve[-50:]) < 0.8 * np.mean(curve[:10])
        # evaluation sequences are not among the training ones
        ev = {"arm": lambda: W.make_planar_arm(B=32, T=30, N=256, L=5, first=1000),
              "clutter": lambda: W.make_clutter_cv(B=32, Tmin=30, Tmax=30, N=256, L=5, first=1000)}[which]()
        j5 = _mean_J(ev, 5)
        jl = _mean_J(ev, 5, p)
        j50 = _mean_J(ev, 50)
        print(f"{which}: mean J plain L5 {j5:.2f}, learned L5 {jl:.2f}, plain L50 {j50:.2f}")
        assert jl > j5
    finally:
        abi.smap_proposal_destroy(p)


def test_forward_wait_that_runs_out_returns_timeout(torch):
    """Every wait of the tensor-core forward is bounded. With stall = 1 the
    MMA-issuing thread first waits on a barrier that nothing completes, so its
    wait runs out before any MMA is issued, then the other warps' waits run
    out: the call reports SMAP_E_TIMEOUT, and the next forward with the
    default limit succeeds and matches a plain forward."""
    p, n_in, n_out = _prop(torch, 3, W.clutter_params(), seed=6)
    try:
        rng = np.random.default_rng(8)
        R = 152 * 128 + 5
        feat = torch.zeros((R, INP), dtype=torch.float32, device="cuda")
        feat[:, :n_in] = torch.from_numpy(rng.normal(0, 1, (R, n_in)).astype(np.float32)).cuda()
        ref = torch.empty((R, n_out), dtype=torch.float32, device="cuda")
        abi.smap_proposal_forward(p, feat, ref)
        disp = torch.full((R, n_out), float("nan"), dtype=torch.float32, device="cuda")
        for wait_ns in (0, 1_000_000):
            with pytest.raises(abi.SmapError) as e:
                abi.smap_debug_proposal_forward(p, feat, disp, wait_ns, stall=1)
            assert e.value.status == abi.SMAP_E_TIMEOUT
        abi.smap_debug_proposal_forward(p, feat, disp, 2_000_000_000, stall=0)
        assert torch.equal(disp, ref)
        disp.fill_(float("nan"))
        abi.smap_proposal_forward(p, feat, disp)
        assert torch.equal(disp, ref)
    finally:
        abi.smap_proposal_destroy(p)


def test_adam_steps_match_oracle(oracle, torch):
    """Two training steps on a one-row set (every minibatch row is that row)
    against the oracle's Adam on the gradients the library reports at the same
    weights: the FP32 master weights agree elementwise to FP32 rounding."""
    p, n_in, n_out = _prop(torch, 4, W.arm_params(), seed=12)
    try:
        rng = np.random.default_rng(4)
        feat = np.zeros((1, INP), np.float32); feat[0, :n_in] = rng.normal(0, 1, n_in)
        targ = np.zeros((1, OUTP), np.float32); targ[0, :n_out] = rng.normal(0, 1, n_out)
        fd, td = torch.from_numpy(feat).cuda(), torch.from_numpy(targ).cuda()
        th0, _ = abi.smap_proposal_get_weights(p)
        lr = 1e-3
        theta = th0.astype(np.float64)
        m = np.zeros_like(theta)
        v = np.zeros_like(theta)
        for step in (1, 2):
            _, g = abi.smap_proposal_loss_grad(p, fd, td)      # gradient at the current weights
            abi.smap_proposal_train(p, fd, td, 1, 1, lr, lr)
            got, _ = abi.smap_proposal_get_weights(p)
            oracle.adam(theta, g.astype(np.float64), m, v, step, lr)
            tol = 2.0 ** -22 * np.abs(theta) + 1e-5 * lr
            bad = np.abs(got - theta) > tol
            assert not np.any(bad), (step, np.flatnonzero(bad)[:8])
            assert np.any(got != th0)
            theta = got.astype(np.float64)     # continue from the library's rounding
    finally:
        abi.smap_proposal_destroy(p)


def _trained_prop(torch, mk_train, seed=9, steps=300):
    """A proposal trained briefly on rows captured from a plain run (so that
    its outputs lie inside the clamp, as a used network's do)."""
    wl = mk_train()
    p, n_in, n_out = _prop(torch, wl.kind, wl.params, seed=seed)
    rows = int(np.sum(wl.T)) * wl.N
    feat = torch.empty((rows, INP), dtype=torch.float32, device="cuda")
    targ = torch.empty((rows, OUTP), dtype=torch.float32, device="cuda")
    with Estimator.from_workload(wl) as est:
        est.run_batch(wl.y, wl.T)
        n = abi.smap_proposal_capture(p, est.h, feat, targ)
    abi.smap_proposal_fit_normalization(p, feat[:n], targ[:n])
    abi.smap_proposal_train(p, feat[:n], targ[:n], steps, 1024, 1e-3, 1e-4)
    return p, n_in, n_out


@pytest.mark.parametrize("which", ["clutter", "arm"])
def test_learned_batched_run_matches_oracle_step_by_step(oracle, torch, which):
    """The learned batched path (rows kernel -> tensor-core network -> one-step
    SVGD kernel, two chains, graph-captured) held to the oracle at every step
    of every sequence, each stage from the GPU's own inputs:
      (i)   x^(0) - u against the oracle's perceptron on the BF16-rounded
            weights, with u and the features recomputed by the oracle from the
            GPU's previous set (within 3e-2 of the displacement spread);
      (ii)  the step's final set against L_learned oracle SVGD iterations from
            the GPU's x^(0) and previous set (1e-3 relative);
      (iii) backpointers, path and J against the oracle's recursion on the
            GPU's sets (identical where the margin exceeds 1e-6, J to 1e-12)."""
    L = 5
    if which == "clutter":
        mk_train = lambda: W.make_clutter_cv(B=8, Tmin=6, Tmax=6, N=48, L=30, first=500)
        wl = W.make_clutter_cv(B=3, Tmin=6, Tmax=6, N=48, L=L)
    else:
        mk_train = lambda: W.make_planar_arm(B=8, T=6, N=48, L=30, first=500)
        wl = W.make_planar_arm(B=3, T=6, N=48, L=L)
    p, n_in, n_out = _trained_prop(torch, mk_train)
    try:
        theta, norm = abi.smap_proposal_get_weights(p)
        B, T, N, d = wl.B, wl.maxT, wl.N, wl.d
        xinit = torch.full((B, T, N, d), float("nan"), dtype=torch.float32, device="cuda")
        with Estimator.from_workload(wl) as est:
            abi.smap_set_proposal(est.h, p, L)
            abi.smap_debug_record_learned_init(est.h, xinit)
            path, J = est.run_batch(wl.y, wl.T)
            abi.smap_debug_record_learned_init(est.h, None)
            hist = est.history()
            psi = est.backpointers()
        xi = xinit.cpu().numpy()
        assert np.all(np.isfinite(xi))
        m = oracle.Model(wl.kind, wl.params)
        Wp = unpack(theta, n_in, n_out)
        mu_in, sd_in = norm[:n_in], norm[INP:INP + n_in]
        mu_out, sd_out = norm[2 * INP:2 * INP + n_out], norm[2 * INP + OUTP:2 * INP + OUTP + n_out]
        got_disp, ref_disp, worst_svgd = [], [], 0.0
        for b in range(B):
            for t in range(1, T + 1):
                z = wl.y[b, t - 1].astype(np.float64)
                prev = wl.x0[b][None, :] if t == 1 else hist[b, t - 2].astype(np.float64)
                fprev = np.array([m.transition(t, v) for v in prev])
                a = fprev[np.zeros(N, int)] if t == 1 else fprev
                u = np.array([a[i] + np.sqrt(m.q) * oracle.normals(wl.seed, b, t, i, d) for i in range(N)])
                f = np.array([oracle.proposal_features(wl.kind, wl.params, u[i], z) for i in range(N)])
                xn = bf16(((f - mu_in) / sd_in).astype(np.float32))
                o = oracle.mlp_forward(n_in, H, n_out, Wp, xn)
                ref_disp.append(np.clip(o, -8.0, 8.0) * sd_out + mu_out)
                got_disp.append(xi[b, t - 1].astype(np.float64) - u)
                # (ii) the SVGD iterations of the step from the GPU's x^(0)
                xo, _ = m.svgd_iters(wl.prior, wl.bw_rule, wl.bw_value, t, z, fprev,
                                     xi[b, t - 1].astype(np.float64), L, wl.step)
                e = float(np.max(np.abs(hist[b, t - 1] - xo)) / max(1.0, np.sqrt(np.mean(xo * xo))))
                worst_svgd = max(worst_svgd, e)
        got_disp, ref_disp = np.concatenate(got_disp), np.concatenate(ref_disp)
        spread = np.std(ref_disp, axis=0).max()
        assert np.max(np.abs(got_disp - ref_disp)) <= 3e-2 * spread
        assert worst_svgd <= 1e-3, worst_svgd
        # (iii) the recursion on the GPU's own sets
        for b in range(B):
            h64, z64 = hist[b].astype(np.float64), wl.y[b].astype(np.float64)
            ref = oracle.viterbi_sets(wl.kind, wl.params, wl.x0[b], h64, z64)
            ok = oracle.viterbi_margins(wl.kind, wl.params, wl.x0[b], h64, z64) > 1e-6
            assert np.array_equal(psi[b][ok], ref["psi"][ok])
            assert J[b] == pytest.approx(ref["J"], rel=1e-12, abs=1e-9)
            assert np.array_equal(path[b], ref["path"].astype(np.float32))
    finally:
        abi.smap_proposal_destroy(p)
