"""Parity of the learned-warm-start kernels with the CPU oracle, and the gain it brings.

The tcgen05 GEMM is compared with the exact FP64 product of the same BF16 operands (the
error of FP32 accumulation over K terms is bounded by K 2^-24 sum|a||b|, taken with a
margin of 4); conversions must match the oracle's BF16 rounding bit for bit; the network's
forward pass, gradients and Adam steps, the warm-start loss and the decoder must match the
oracle run on the same BF16 values (normwise 1e-3: both sides round activations to BF16 at
the same points, so only accumulation order differs, which flips a rounding rarely; the
forward output and the gradients also element by element: within worst-case bounds derived
from the FP32 accumulation and BF16 rounding of every layer, and within 1e-2 of the largest
magnitude).
The last test trains the warm start on a small family and checks that held-out members
converge in fewer iterations than from the origin, to the same objective.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import learned as OL
import qpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2507_02470_gb300 as p
    p.build()
    from paper_2507_02470_gb300 import learned as L
    return torch, p, L


def bf16_tensor(torch, a, ld=None):
    """CUDA bfloat16 tensor with the oracle's rounding of a (rows x cols), row stride ld."""
    a = np.atleast_2d(a)
    rows, cols = a.shape
    ld = ld or (cols + 7) // 8 * 8
    bits = np.zeros((rows, ld), dtype=np.uint16)
    bits[:, :cols] = OL.bf16_bits(a)
    t = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    return t, OL.from_bf16_bits(bits[:, :cols])


def normrel(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


U16 = 2.0 ** -8    # unit roundoff of BF16 (8 significant bits)
U32 = 2.0 ** -24   # unit roundoff of FP32, the GEMMs' accumulators


def mlp_bounds(Ws, bs, hs, dY, B):
    """Element-wise bounds on |GPU - oracle| for the forward output and the gradients, from the
    arithmetic alone: both sides take the same BF16 inputs and weights; a GEMM over K terms in
    FP32 differs from the exact sum by at most 4 K U32 sum|a||b|; a value rounded to BF16 on both
    sides from inputs e apart differs by at most e + U16 (|a| + |b|); ReLU is 1-Lipschitz.  A
    ReLU mask may differ only where the oracle's input is within its bound of 0 (there the whole
    value counts as error).  Loose on purpose: a rounding that flips rarely stays far inside."""
    L = len(Ws)
    Wb = [np.abs(OL.bf16_round(w)) for w in Ws]
    e = np.zeros_like(hs[0])
    eh = [e]
    ez = None
    for l in range(L):
        K = Ws[l].shape[1]
        # the GEMM's accumulation, then the FP32 bias add (and, for the output, its FP32 store)
        az = (np.abs(hs[l]) + e) @ Wb[l].T
        ez = e @ Wb[l].T + 4 * K * U32 * az + 2 * U32 * (az + np.abs(bs[l]))
        if l + 1 < L:
            e = ez + U16 * (2 * hs[l + 1] + ez)
            eh.append(e)
    eY = ez
    # backward: dZ of the last layer is the same BF16 rounding of the same dY on both sides
    dZ = OL.bf16_round(dY)
    edZ = np.zeros_like(dZ)
    eW, eb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        aZ, aH = np.abs(dZ), np.abs(hs[l])
        eW[l] = edZ.T @ (aH + eh[l]) + aZ.T @ eh[l] + 4 * B * U32 * ((aZ + edZ).T @ (aH + eh[l]))
        eb[l] = edZ.sum(axis=0) + 4 * B * U32 * (aZ + edZ).sum(axis=0)
        if l == 0:
            break
        K = Ws[l].shape[0]
        dX = dZ @ OL.bf16_round(Ws[l])
        edX = edZ @ Wb[l] + 4 * K * U32 * ((aZ + edZ) @ Wb[l])
        unsure = hs[l] <= eh[l]
        dZn = OL.bf16_round(dX * (hs[l] > 0))
        edZ = np.where(unsure, np.abs(dX) + edX + U16 * (np.abs(dX) + edX),
                       edX + U16 * (2 * np.abs(dZn) + edX))
        dZ = dZn
    return eY, eW, eb


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 64, 1), (256, 384, 1024, 1), (200, 100, 150, 1),
                                          (300, 50, 700, 3), (1, 1, 1, 1), (129, 65, 8, 1), (640, 256, 4096, 16),
                                          (256, 640, 192, 1), (300, 1000, 300, 2), (130, 513, 4000, 0)])
def test_gemm_matches_exact_product(env, M, N, K, splits):
    torch, p, L = env
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A, Av = bf16_tensor(torch, rng.standard_normal((M, K)))
    B, Bv = bf16_tensor(torch, rng.standard_normal((N, K)))
    A = A[:, :K]
    B = B[:, :K]
    out = torch.full((M, N + 5), float("nan"), dtype=torch.float32, device="cuda")[:, :N]
    L.gemm_bf16(A, B, out=out, splits=splits)
    L.check()
    ref = Av @ Bv.T
    bound = 4 * K * 2.0 ** -24 * (np.abs(Av) @ np.abs(Bv).T) + 1e-30
    got = out.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


def test_gemm_rejects_bad_arguments(env):
    torch, p, L = env
    from paper_2507_02470_gb300 import HPRQPError
    A = torch.zeros(8, 12, dtype=torch.bfloat16, device="cuda")      # row stride 12: not 16-byte rows
    with pytest.raises(HPRQPError):
        L.gemm_bf16(A, A)


def test_cast_is_bit_exact(env):
    torch, p, L = env
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, 37)) * 10.0 ** rng.integers(-30, 30, (5, 37))
    x[0, 0], x[1, 1], x[2, 2] = np.inf, -np.inf, np.nan
    sub = rng.standard_normal(37)
    xt = torch.from_numpy(x).cuda()
    nrm = torch.zeros(5, dtype=torch.float64, device="cuda")
    out = L.cast_bf16(xt, sub=torch.from_numpy(sub).cuda(), scale=0.5, ld=48, rownorm2=nrm)
    bits = out.view(torch.int16).cpu().numpy().view(np.uint16)
    v = (x - sub[None, :]) * 0.5
    assert np.array_equal(bits[:, :37], OL.bf16_bits(v))
    assert np.all(bits[:, 37:] == 0)
    vv = np.where(np.isfinite(v), v, 0.0)
    assert np.allclose(nrm.cpu().numpy(), np.sum(vv * vv, axis=1), rtol=1e-12)
    out32 = L.cast_bf16(torch.from_numpy(x.astype(np.float32)).cuda())
    bits32 = out32.view(torch.int16).cpu().numpy().view(np.uint16)[:, :37]
    assert np.array_equal(bits32, OL.bf16_bits(x.astype(np.float32)))


def test_row_stats_and_col_mean(env):
    torch, p, L = env
    import ctypes as C
    lib = p.lib()
    rng = np.random.default_rng(4)
    F = (3.0 + 2.0 * rng.standard_normal((9, 1001))).astype(np.float32)
    Ft = torch.from_numpy(F).cuda()
    mean = torch.empty(9, dtype=torch.float32, device="cuda")
    istd = torch.empty(9, dtype=torch.float32, device="cuda")
    assert lib.hprqp_row_stats(Ft.data_ptr(), 9, 1001, 1001, C.c_float(1e-12), mean.data_ptr(), istd.data_ptr(),
                               None) == 0
    mu, isd = OL.row_stats(F.astype(np.float64), 1e-12)
    assert np.allclose(mean.cpu().numpy(), mu, rtol=1e-6) and np.allclose(istd.cpu().numpy(), isd, rtol=1e-6)
    Z = rng.standard_normal((33, 70))
    Zt = torch.from_numpy(Z).cuda()
    m = torch.empty(70, dtype=torch.float64, device="cuda")
    assert lib.hprqp_col_mean_f64(Zt.data_ptr(), 33, 70, 70, m.data_ptr(), None) == 0
    assert np.allclose(m.cpu().numpy(), Z.mean(axis=0), rtol=1e-13, atol=1e-15)


def _random_net(rng, dims):
    Ws = [rng.standard_normal((dims[l + 1], dims[l])) * math.sqrt(2.0 / dims[l]) for l in range(len(dims) - 1)]
    bs = [0.1 * rng.standard_normal(dims[l + 1]) for l in range(len(dims) - 1)]
    return [w.astype(np.float32).astype(np.float64) for w in Ws], [b.astype(np.float32).astype(np.float64) for b in bs]


@pytest.mark.parametrize("dims,B", [([72, 200, 136, 65], 50), ([512, 1024, 1024, 257], 256)])
def test_mlp_forward_backward_adam_match_oracle(env, dims, B):
    torch, p, L = env
    rng = np.random.default_rng(len(dims) + B)
    Ws, bs = _random_net(rng, dims)
    net = L.MLP(dims, max_batch=B)
    for l in range(len(Ws)):
        net.set_layer(l, Ws[l], bs[l])
    X, Xv = bf16_tensor(torch, rng.standard_normal((B, dims[0])))
    Y = net.forward(X)
    Yref, hs = OL.mlp_forward(Ws, bs, Xv)
    assert normrel(Y.cpu().numpy(), Yref) <= 1e-3
    dY = rng.standard_normal((B, dims[-1])) / B
    net.backward(torch.from_numpy(dY.astype(np.float32)).cuda())
    dY64 = dY.astype(np.float32).astype(np.float64)
    gW, gb = OL.mlp_backward(Ws, hs, dY64)
    eY, eW, eb = mlp_bounds(Ws, bs, hs, dY64, B)
    Yg = Y.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Yg - Yref) <= eY), np.max(np.abs(Yg - Yref) / (eY + 1e-300))
    # the worst-case bound above assumes every rounding flips; in fact few do, so every output
    # element also stays within 1e-2 of the output's largest magnitude
    assert np.max(np.abs(Yg - Yref)) <= 1e-2 * np.max(np.abs(Yref))
    for l in range(len(Ws)):
        w, b = net.get_grad(l)
        assert normrel(w, gW[l]) <= 1e-3, l
        assert normrel(b, gb[l]) <= 1e-3, l
        w, b = np.asarray(w, dtype=np.float64), np.asarray(b, dtype=np.float64)
        assert np.all(np.abs(w - gW[l]) <= eW[l]), (l, np.max(np.abs(w - gW[l]) / (eW[l] + 1e-300)))
        assert np.all(np.abs(b - gb[l]) <= eb[l]), (l, np.max(np.abs(b - gb[l]) / (eb[l] + 1e-300)))
        assert np.max(np.abs(w - gW[l])) <= 1e-2 * np.max(np.abs(gW[l])), l
        assert np.max(np.abs(b - gb[l])) <= 1e-2 * np.max(np.abs(gb[l])), l
    # three Adam steps on the same gradients
    Wr = [w.copy() for w in Ws]
    br = [b.copy() for b in bs]
    mom = [[np.zeros_like(w), np.zeros_like(w), np.zeros_like(b), np.zeros_like(b)] for w, b in zip(Ws, bs)]
    g_gpu = [net.get_grad(l) for l in range(len(Ws))]
    for t in range(1, 4):
        net.adam(lr=1e-3)
        for l in range(len(Ws)):
            gw, gbb = (g.astype(np.float64) for g in g_gpu[l])
            Wr[l], mom[l][0], mom[l][1] = OL.adam(Wr[l], mom[l][0], mom[l][1], gw, t, 1e-3, 0.9, 0.999, 1e-8)
            br[l], mom[l][2], mom[l][3] = OL.adam(br[l], mom[l][2], mom[l][3], gbb, t, 1e-3, 0.9, 0.999, 1e-8)
    for l in range(len(Ws)):
        w, b = net.get_layer(l)
        assert np.max(np.abs(w - Wr[l])) <= 1e-6 + 1e-5 * np.max(np.abs(Wr[l])), l
        assert np.max(np.abs(b - br[l])) <= 1e-6 + 1e-5 * np.max(np.abs(br[l])), l
    L.check()
    net.close()


def test_ws_loss_and_decode_match_oracle(env):
    torch, p, L = env
    import ctypes as C
    lib = p.lib()
    rng = np.random.default_rng(7)
    B, r, D, extra = 19, 40, 333, 5
    Out = rng.standard_normal((B, 1 + r + extra)).astype(np.float32)
    Phi, Phiv = bf16_tensor(torch, rng.standard_normal((D, r)) / math.sqrt(r))
    mu = rng.standard_normal(D)
    Zs = mu[None, :] + rng.standard_normal((B, D))
    G = (Phiv.T @ Phiv).astype(np.float32)
    R = (Phiv.T @ (Zs - mu[None, :]).T).astype(np.float32)
    dd = np.sum((Zs - mu[None, :]) ** 2, axis=1)
    s = rng.standard_normal(B).astype(np.float32)
    alpha, E, w_sigma, s_mean, s_istd = 0.3, float(D), 1.5, 0.2, 2.0
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dO = torch.zeros(B, 1 + r + extra, dtype=torch.float32, device="cuda")
    loss = torch.zeros(2, dtype=torch.float32, device="cuda")
    Og, Gg, Rg, ddg, sg = t(Out), t(G), t(R), t(dd), t(s)
    assert lib.hprqp_ws_loss(Og.data_ptr(), Og.stride(0), B, r, Gg.data_ptr(), Rg.data_ptr(), B, ddg.data_ptr(),
                             sg.data_ptr(), C.c_float(s_mean), C.c_float(s_istd), C.c_float(alpha), C.c_float(E),
                             C.c_float(w_sigma), dO.data_ptr(), dO.stride(0), 1 + r + extra, loss.data_ptr(),
                             None) == 0
    dref, ls, ll = OL.ws_loss(Out, G.astype(np.float64), R.astype(np.float64), dd, s.astype(np.float64), alpha, E,
                              w_sigma, r, s_mean, s_istd)
    assert normrel(dO.cpu().numpy(), dref) <= 1e-5
    assert abs(loss[0].item() - ls) <= 1e-5 * abs(ls) and abs(loss[1].item() - ll) <= 1e-5 * abs(ll)
    lo = np.full(D, -1.0)
    hi = np.full(D, 1.0)
    lo[::3] = -np.inf
    Z = torch.empty(B, D + 3, dtype=torch.float64, device="cuda")
    sig = torch.empty(B, dtype=torch.float64, device="cuda")
    work = torch.empty(D * B, dtype=torch.float32, device="cuda")
    assert lib.hprqp_ws_decode(Phi.data_ptr(), Phi.stride(0), D, r, Og.data_ptr(), Og.stride(0), B, C.c_float(alpha),
                               C.c_float(s_mean), C.c_float(s_istd), t(mu).data_ptr(), t(lo).data_ptr(),
                               t(hi).data_ptr(), work.data_ptr(), Z.data_ptr(), Z.stride(0), sig.data_ptr(),
                               None) == 0
    Zref = OL.decode(Phiv, mu, OL.bf16_round(Out[:, 1:1 + r]), alpha, lo, hi)
    got = Z.cpu().numpy()[:, :D]
    assert np.max(np.abs(got - Zref)) <= 1e-5 * (1 + np.max(np.abs(Zref)))
    assert np.allclose(sig.cpu().numpy(), OL.sigma0(Out, s_mean, s_istd), rtol=1e-6)
    L.check()


def test_learned_warm_start_reduces_iterations(env):
    torch, p, L = env
    base = qpgen.param_family_base(n=4000, m=2000, seed=5)
    Ntr, Nte = 320, 24
    Ctr, Utr = qpgen.ws_family_data(base, range(Ntr))
    Cte, Ute = qpgen.ws_family_data(base, range(100_000, 100_000 + Nte))
    Z = torch.empty(Ntr, base.n + base.m, dtype=torch.float64, device="cuda")
    tr = L.solve_members(base, lambda a, b: (Ctr[a:b], Utr[a:b]), Ntr, Z=Z, workers=2)
    assert all(s == "converged" for s in tr["status"])
    ws = L.LearnedWarmStart(base.n, base.m, base.L, base.U, base.l, base.u, d0=128, hidden=(256, 256), r=32,
                            seed=1, max_batch=64, chunk=128)
    rep = ws.fit((Ctr, Utr), Z, tr["sigma"], epochs=60, batch=64, lr=1e-3)
    assert rep.loss_latent[-1] < rep.latent_baseline      # better than decoding to mu alone
    assert rep.loss_sigma[-1] < rep.loss_sigma[0]
    Z0, sig0 = ws.predict(Cte, Ute)
    L.check()
    # held-out members: from the origin with the sigma0 rule, and from the learned start
    te = lambda a, b: (Cte[a:b], Ute[a:b])
    cold = L.solve_members(base, te, Nte, lam=tr["lambda"])
    warm = L.solve_members(base, te, Nte, lam=tr["lambda"], starts=(Z0.cpu().numpy(), sig0.cpu().numpy()))
    assert all(s == "converged" for s in cold["status"] + warm["status"])
    assert np.all(np.abs(warm["pobj"] - cold["pobj"]) <= 1e-6 * np.maximum(1.0, np.abs(cold["pobj"])))
    assert warm["iters"].mean() < 0.9 * cold["iters"].mean(), (warm["iters"].mean(), cold["iters"].mean())
    ws.close()


def test_warm_start_falls_back_to_cold(env):
    """A rejected prediction (non-finite) is replaced by the cold start, and the member still
    converges to the cold start's objective."""
    torch, p, L = env
    base = qpgen.param_family_base(n=2000, m=1000, seed=7)
    C, U = qpgen.ws_family_data(base, range(3))
    data = lambda a, b: (C[a:b], U[a:b])
    cold = L.solve_members(base, data, 3)
    Z0 = np.zeros((3, base.n + base.m))
    Z0[1, 5] = np.nan
    warm = L.solve_members(base, data, 3, starts=(Z0, np.ones(3)), lam=cold["lambda"])
    assert warm["fallbacks"] == 1
    assert all(s == "converged" for s in warm["status"])
    assert np.allclose(warm["pobj"], cold["pobj"], rtol=1e-6)
