"""GPU tests of the product building block D = alpha X Y^T + beta C + gamma I (C ABI).

Reference: the same FP32/FP64 inputs multiplied in FP64 by NumPy on the host.
Shapes span several 128 x 256 tiles with ragged M, N and K tails.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# relative Frobenius bounds for K <= 4096 with O(1) entries:
#  3xTF32 / FFMA carry FP32 rounding (~ sqrt(K) 2^-24), 1xTF32 carries 2^-11 per operand
TOL = {"simt": 2e-6, "3xtf32": 4e-6, "tf32": 3e-3, "auto": 4e-6}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _mat(rng, rows, cols, ld=None, dtype=np.float32):
    ld = cols if ld is None else ld
    A = np.zeros((rows, ld), dtype=dtype)
    A[:, :cols] = rng.standard_normal((rows, cols))
    return A


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("engine", ["simt", "3xtf32", "tf32"])
@pytest.mark.parametrize("M,N,K", [(128, 256, 32), (300, 200, 130), (1024, 1024, 1024),
                                   (777, 513, 2049)])
def test_gemm_f32_plain(cuda, cdmpt_lib, engine, M, N, K):
    import torch
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    ld = (K + 3) // 4 * 4
    X = _mat(rng, M, K, ld)
    Y = _mat(rng, N, K, ld)
    D = torch.zeros((M, (N + 3) // 4 * 4), dtype=torch.float32, device=cuda)
    cdmpt_lib.gemm_f32(_t(X, cuda), _t(Y, cuda), D, engine=engine, M=M, Ncols=N, K=K)
    torch.cuda.synchronize()
    ref = X[:, :K].astype(np.float64) @ Y[:, :K].astype(np.float64).T
    assert _rel(D.cpu().numpy()[:, :N].astype(np.float64), ref) < TOL[engine]


@pytest.mark.parametrize("engine", ["simt", "3xtf32", "tf32"])
@pytest.mark.parametrize("Nb", [160, 150])
def test_gemm_f32_epilogue(cuda, cdmpt_lib, engine, Nb):
    """alpha, beta C, gamma on block diagonals, transposed block placement and the fused dot.
    Nb = 150: the diagonal blocks start inside the epilogue's 32-row store blocks."""
    import torch
    rng = np.random.default_rng(5)
    blocks = 2
    M, N, K = Nb * blocks, Nb, Nb
    ldk = (K + 3) // 4 * 4      # operand rows 16-byte aligned (zero padding adds nothing)
    X = _mat(rng, M, K, ld=ldk)
    Y = _mat(rng, N, K, ld=ldk)
    C = _mat(rng, M, N)
    E = _mat(rng, M, N)
    alpha, beta, gamma = -1.25, 2.0, 0.75
    acc = X.astype(np.float64) @ Y.astype(np.float64).T
    for trans in (0, Nb):
        ref = np.empty((M, N))
        for b in range(blocks):
            blk = alpha * acc[b * Nb:(b + 1) * Nb] + gamma * np.eye(Nb)
            if trans:
                ref[b * Nb:(b + 1) * Nb] = blk.T + beta * C[b * Nb:(b + 1) * Nb]
            else:
                ref[b * Nb:(b + 1) * Nb] = blk + beta * C[b * Nb:(b + 1) * Nb]
        D = torch.zeros((M, N), dtype=torch.float32, device=cuda)
        dot = torch.zeros(1, dtype=torch.float64, device=cuda)
        cdmpt_lib.gemm_f32(_t(X, cuda), _t(Y, cuda), D, alpha=alpha, beta=beta, C=_t(C, cuda),
                           gamma=gamma, diag_block=Nb, trans_block=trans, dot=dot, E=_t(E, cuda),
                           engine=engine)
        torch.cuda.synchronize()
        got = D.cpu().numpy().astype(np.float64)
        assert _rel(got, ref) < TOL[engine], trans
        assert abs(dot.item() - np.sum(got * E)) < 1e-5 * np.sum(np.abs(got * E))
        # self dot (E = D)
        dot.zero_()
        cdmpt_lib.gemm_f32(_t(X, cuda), _t(Y, cuda), D, alpha=alpha, beta=beta, C=_t(C, cuda),
                           gamma=gamma, diag_block=Nb, trans_block=trans, dot=dot, engine=engine)
        torch.cuda.synchronize()
        got = D.cpu().numpy().astype(np.float64)
        assert abs(dot.item() - np.sum(got * got)) < 1e-5 * np.sum(got * got)


def test_gemm_f32_in_place_accumulate(cuda, cdmpt_lib):
    """C may alias D: D = X Y^T + D."""
    import torch
    rng = np.random.default_rng(9)
    X = _mat(rng, 256, 256)
    Y = _mat(rng, 256, 256)
    C = _mat(rng, 256, 256)
    D = _t(C, cuda).clone()
    cdmpt_lib.gemm_f32(_t(X, cuda), _t(Y, cuda), D, beta=1.0, C=D, engine="3xtf32")
    torch.cuda.synchronize()
    ref = X.astype(np.float64) @ Y.astype(np.float64).T + C
    assert _rel(D.cpu().numpy().astype(np.float64), ref) < TOL["3xtf32"]


def test_gemm_f64(cuda, cdmpt_lib):
    import torch
    rng = np.random.default_rng(3)
    M, N, K = 100, 70, 90
    X = _mat(rng, M, K, dtype=np.float64)
    Y = _mat(rng, N, K, dtype=np.float64)
    C = _mat(rng, M, N, dtype=np.float64)
    D = torch.zeros((M, N), dtype=torch.float64, device=cuda)
    dot = torch.zeros(1, dtype=torch.float64, device=cuda)
    cdmpt_lib.gemm_f64(_t(X, cuda), _t(Y, cuda), D, alpha=0.5, beta=-1.0, C=_t(C, cuda),
                       gamma=3.0, dot=dot)
    torch.cuda.synchronize()
    ref = 0.5 * X @ Y.T - C
    ref[np.arange(N), np.arange(N)] += 3.0
    got = D.cpu().numpy()
    assert _rel(got, ref) < 1e-14
    assert abs(dot.item() - np.sum(got * got)) < 1e-12 * np.sum(got * got)


@pytest.mark.parametrize("M,N,K", [(100, 70, 90), (300, 200, 130), (1024, 1024, 1024),
                                   (777, 513, 2049)])
def test_gemm_f64_tensor_core_matches_fp64(cuda, cdmpt_lib, M, N, K):
    """FP64 Ozaki product (seven BF16 digits per element, cdmpt_gemm_f64_tc) against NumPy's
    FP64 product: rows spread over 2^-30 .. 2^30 (the per-row powers of two of the slicing),
    one all-zero row, ragged M, N and K (partial tiles, a K tail beyond the last 32-block)."""
    import torch
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    X = _mat(rng, M, K, dtype=np.float64) * np.exp2(rng.integers(-30, 31, size=M))[:, None]
    Y = _mat(rng, N, K, dtype=np.float64) * np.exp2(rng.integers(-30, 31, size=N))[:, None]
    X[M // 3] = 0.0
    C = _mat(rng, M, N, dtype=np.float64)
    D = torch.zeros((M, N), dtype=torch.float64, device=cuda)
    dot = torch.zeros(1, dtype=torch.float64, device=cuda)
    cdmpt_lib.gemm_f64(_t(X, cuda), _t(Y, cuda), D, alpha=0.5, beta=-1.0, C=_t(C, cuda),
                       gamma=3.0, dot=dot, engine="tc")
    torch.cuda.synchronize()
    P = X @ Y.T
    ref = 0.5 * P - C
    ref[np.arange(min(M, N)), np.arange(min(M, N))] += 3.0
    got = D.cpu().numpy()
    # elementwise against the scale of the terms (row and column maxima of |X| |Y|^T)
    scale = 0.5 * np.abs(X).max(axis=1)[:, None] * np.abs(Y).max(axis=1)[None, :] * K
    assert np.all(np.abs(got - ref) <= 2.0 ** -44 * scale + 4e-16 * np.abs(ref) + 1e-300)
    assert _rel(got, ref) < 1e-13
    assert abs(dot.item() - np.sum(got * got)) < 1e-12 * np.sum(got * got)


def test_gemm_f64_tensor_core_epilogue(cuda, cdmpt_lib):
    """alpha, beta C, gamma on block diagonals, transposed block placement and the fused dot
    with E on the FP64 tensor-core engine."""
    import torch
    rng = np.random.default_rng(11)
    Nb, blocks = 160, 2
    M, N, K = Nb * blocks, Nb, Nb
    X = _mat(rng, M, K, dtype=np.float64)
    Y = _mat(rng, N, K, dtype=np.float64)
    C = _mat(rng, M, N, dtype=np.float64)
    E = _mat(rng, M, N, dtype=np.float64)
    alpha, beta, gamma = -1.25, 2.0, 0.75
    acc = X @ Y.T
    for trans in (0, Nb):
        ref = np.empty((M, N))
        for b in range(blocks):
            blk = alpha * acc[b * Nb:(b + 1) * Nb] + gamma * np.eye(Nb)
            ref[b * Nb:(b + 1) * Nb] = (blk.T if trans else blk) + beta * C[b * Nb:(b + 1) * Nb]
        D = torch.zeros((M, N), dtype=torch.float64, device=cuda)
        dot = torch.zeros(1, dtype=torch.float64, device=cuda)
        cdmpt_lib.gemm_f64(_t(X, cuda), _t(Y, cuda), D, alpha=alpha, beta=beta, C=_t(C, cuda),
                           gamma=gamma, diag_block=Nb, trans_block=trans, dot=dot, E=_t(E, cuda),
                           engine="tc")
        torch.cuda.synchronize()
        got = D.cpu().numpy()
        assert _rel(got, ref) < 1e-13, trans
        assert abs(dot.item() - np.sum(got * E)) < 1e-12 * np.sum(np.abs(got * E))


def test_gemm_rejects_misaligned_ld(cuda, cdmpt_lib):
    import torch
    X = torch.zeros((64, 66), dtype=torch.float32, device=cuda)
    D = torch.zeros((64, 64), dtype=torch.float32, device=cuda)
    with pytest.raises(cdmpt_lib.CdmptError):
        cdmpt_lib.gemm_f32(X, X, D, engine="tf32", K=66)


def test_spectral_bounds(cuda, cdmpt_lib):
    """Gershgorin interval: equals the disc formula and contains every eigenvalue."""
    import torch
    import synthetic as syn
    for p in (syn.workload("chain64"), syn.cubic_lattice((7, 7, 7), seed=2)):
        H = torch.from_numpy(p.H0).to(cuda)
        b = cdmpt_lib.spectral_bounds(H).cpu().numpy()
        rad = np.abs(p.H0).sum(1) - np.abs(np.diag(p.H0))
        lo, hi = np.min(np.diag(p.H0) - rad), np.max(np.diag(p.H0) + rad)
        assert abs(b[0] - lo) < 1e-12 and abs(b[1] - hi) < 1e-12
        ev = np.linalg.eigvalsh(p.H0)
        assert b[0] <= ev[0] + 1e-12 and ev[-1] <= b[1] + 1e-12


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 200, 136), (1024, 1024, 1024),
                                   (777, 513, 2056)])
def test_gemm_bf16(cuda, cdmpt_lib, M, N, K):
    """BF16 engine (kind::f16, FP32 accumulation) on operands rounded to BF16 inside the call:
    close to the exact FP64 product of the BF16-rounded inputs, and within BF16 rounding of
    the FP32 product."""
    import torch
    rng = np.random.default_rng(M + 5 * N + 11 * K)
    ld = (K + 7) // 8 * 8
    X = _mat(rng, M, K, ld)
    Y = _mat(rng, N, K, ld)
    dev = torch.device("cuda")
    D = torch.zeros((M, N), dtype=torch.float32, device=dev)
    cdmpt_lib.gemm_f32(_t(X, dev), _t(Y, dev), D, gamma=0.5, engine="bf16", M=M, Ncols=N, K=K)
    torch.cuda.synchronize()
    Xb = torch.from_numpy(X[:, :K]).to(torch.bfloat16).double().numpy()
    Yb = torch.from_numpy(Y[:, :K]).to(torch.bfloat16).double().numpy()
    ref_b = Xb @ Yb.T + 0.5 * np.eye(M, N)
    ref = X[:, :K].astype(np.float64) @ Y[:, :K].astype(np.float64).T + 0.5 * np.eye(M, N)
    got = D.cpu().numpy().astype(np.float64)
    assert _rel(got, ref_b) < 4e-5     # FP32 accumulation in TMEM over K
    assert _rel(got, ref) < 1e-2


def test_gemm_bf16_rejects_unaligned_ld(cuda, cdmpt_lib):
    import torch
    X = torch.zeros((64, 36), dtype=torch.float32, device="cuda")
    D = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(cdmpt_lib.CdmptError):
        cdmpt_lib.gemm_f32(X, X, D, engine="bf16", K=36)


@pytest.mark.parametrize("engine", ["3xtf32", "tf32", "bf16"])
@pytest.mark.parametrize("N", [128, 300, 1024, 1100])
def test_gemm_symmetric_result(cuda, cdmpt_lib, engine, N):
    """trans_block = -1 (symmetric result): only upper-triangular tiles are computed and
    mirrored. For commuting symmetric factors (Z and Z^3) with symmetric C and E the result
    equals the full product within the engine's tolerance, is exactly symmetric, and the
    fused dot counts both halves."""
    import torch
    rng = np.random.default_rng(N + len(engine))
    ld = (N + 7) // 8 * 8
    Z = rng.standard_normal((N, N)) / np.sqrt(N)
    Z = 0.5 * (Z + Z.T)
    Y = Z @ Z @ Z
    S = rng.standard_normal((N, N))
    S = 0.5 * (S + S.T)
    E = rng.standard_normal((N, N))
    E = 0.5 * (E + E.T)

    def pad(A):
        B = np.zeros((N, ld), dtype=np.float32)
        B[:, :N] = A
        return torch.from_numpy(B).cuda()

    dev = torch.device("cuda")
    D = torch.zeros((N, ld), dtype=torch.float32, device=dev)
    dot = torch.zeros(1, dtype=torch.float64, device=dev)
    cdmpt_lib.gemm_f32(pad(Z), pad(Y), D, alpha=-2.0, beta=0.5, C=pad(S), gamma=0.25,
                       trans_block=-1, dot=dot, E=pad(E), engine=engine, M=N, Ncols=N, K=N)
    torch.cuda.synchronize()
    got = D.cpu().numpy()[:, :N].astype(np.float64)
    Zf = Z.astype(np.float32).astype(np.float64)
    Yf = Y.astype(np.float32).astype(np.float64)
    ref = -2.0 * Zf @ Yf.T + 0.5 * S.astype(np.float32) + 0.25 * np.eye(N)
    tol = {"3xtf32": 4e-6, "tf32": 3e-3, "bf16": 1e-2}[engine]
    assert np.array_equal(got, got.T)
    assert _rel(got, ref) < tol
    want = float(np.sum(got * E.astype(np.float32)))
    assert abs(float(dot.item()) - want) < 1e-5 * max(1.0, abs(want))


def _pair(v):
    """FP64 values stored as an FP32 pair (hi, lo); returns hi, lo and their exact FP64 sum."""
    hi = v.astype(np.float32)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    return hi, lo, hi.astype(np.float64) + lo.astype(np.float64)


def _pair_mat(rng, rows, cols, ld):
    """Normal entries with row magnitudes spread over 2^-20 .. 2^20 (the per-row powers of two
    of the slicing) and one all-zero row."""
    v = np.zeros((rows, ld))
    v[:, :cols] = rng.standard_normal((rows, cols))
    v[:, :cols] *= np.exp2(rng.integers(-20, 21, size=rows))[:, None]
    v[rows // 2, :] = 0.0
    return _pair(v)


@pytest.mark.parametrize("M,N,K", [(256, 128, 64), (300, 200, 130), (1024, 1024, 1024),
                                   (777, 513, 2049), (2048, 2048, 4096)])
def test_gemm_pair_matches_fp64(cuda, cdmpt_lib, M, N, K):
    """Ozaki-sliced product of FP32 pairs against the FP64 product of the same values. Five
    8-bit digits per row carry the row's values to 2^-39 of its power of two, so an element's
    error is a sum of K such terms of random sign: it stays within 2^-35 sqrt(K) max|x_i.|
    max|y_j.| (with four digits the observed maximum was 2^-29.6 sqrt(K)), and the whole
    product within 3e-11 relative (Frobenius) - far below FP32 (6e-8 per operand), which no
    FP32-accumulating product reaches."""
    import torch
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    ld = (K + 7) // 8 * 8
    Xh, Xl, X = _pair_mat(rng, M, K, ld)
    Yh, Yl, Y = _pair_mat(rng, N, K, ld)
    ldd = (N + 7) // 8 * 8
    D = torch.zeros((M, ldd), dtype=torch.float32, device=cuda)
    Dl = torch.zeros_like(D)
    cdmpt_lib.gemm_pair(_t(Xh, cuda), _t(Xl, cuda), _t(Yh, cuda), _t(Yl, cuda), D, Dl, K=K)
    torch.cuda.synchronize()
    got = D.cpu().numpy()[:, :N].astype(np.float64) + Dl.cpu().numpy()[:, :N].astype(np.float64)
    ref = X[:, :K] @ Y[:, :K].T
    scale = np.abs(X[:, :K]).max(axis=1)[:, None] * np.abs(Y[:, :K]).max(axis=1)[None, :]
    bound = 2.0 ** -35 * np.sqrt(K) * scale
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / np.maximum(bound, 1e-300)))
    assert _rel(got, ref) < 3e-11, _rel(got, ref)
    assert np.all(got[M // 2] == 0.0) and np.all(got[:, N // 2] == 0.0)


def test_gemm_pair_step_residual(cuda, cdmpt_lib):
    """The residual of one recursion step in correction form, R = 2 Z - Z' - Z' W with
    W = Z Z and Z' = 2 Z (I + W)^-1, from pair-stored operands. R cancels to the rounding of
    the pairs (about 2^-48 of |Z|), so the computed R shows the product's own error, which
    must stay below 1e-11 |Z'| |W| (split-TF32 products leave about 1e-7)."""
    import torch
    rng = np.random.default_rng(11)
    N = 1000
    ld = 1008
    A = rng.standard_normal((N, N)) / np.sqrt(N)
    Z = 0.45 * (A + A.T)
    Zh, Zl, Zp = _pair(np.pad(Z, ((0, 0), (0, ld - N))))
    W = Zp[:, :N] @ Zp[:, :N].T
    Wh, Wl, Wp = _pair(np.pad(W, ((0, 0), (0, ld - N))))
    Zn = 2.0 * np.linalg.solve(np.eye(N) + Wp[:, :N], Zp[:, :N])
    Zn = 0.5 * (Zn + Zn.T)
    Znh, Znl, Znp = _pair(np.pad(Zn, ((0, 0), (0, ld - N))))
    R = torch.zeros((N, ld), dtype=torch.float32, device=cuda)
    t = lambda a: _t(a, cuda)
    cdmpt_lib.gemm_pair(t(Znh), t(Znl), t(Wh), t(Wl), R, None, alpha=-1.0, b1=2.0,
                        C1=(t(Zh), t(Zl)), b2=-1.0, C2=(t(Znh), t(Znl)), K=N)
    torch.cuda.synchronize()
    ref = 2.0 * Zp[:, :N] - Znp[:, :N] - Znp[:, :N] @ Wp[:, :N].T
    err = np.abs(R.cpu().numpy()[:, :N].astype(np.float64) - ref).max()
    assert err < 1e-11 * np.abs(Znp).max() * np.abs(Wp).sum(axis=1).max(), err


@pytest.mark.parametrize("N", [300, 1024, 1100])
def test_gemm_pair_symmetric_result(cuda, cdmpt_lib, N):
    """sym = 1 (Y is X): only the output tiles that meet the upper triangle are computed and
    mirrored. The result W = X X^T - I (the right side I - Z_n^2 of dP0/dmu, negated) and its
    TF32 split must equal the full product's (the same element sums, written twice) and be
    exactly symmetric, for N not a multiple of the 256 x 96 tiles."""
    import torch
    rng = np.random.default_rng(N)
    ld = (N + 7) // 8 * 8
    A = rng.standard_normal((N, N)) / np.sqrt(N)
    Zh, Zl, Zp = _pair(np.pad(0.5 * (A + A.T), ((0, 0), (0, ld - N))))
    t = lambda a: _t(a, cuda)
    outs = []
    for sym in (False, True):
        D = torch.zeros((N, ld), dtype=torch.float32, device=cuda)
        Dl = torch.zeros_like(D)
        Xh, Xl = t(Zh), t(Zl)
        cdmpt_lib.gemm_pair(Xh, Xl, Xh, Xl, D, Dl, K=N, sym=sym)
        torch.cuda.synchronize()
        outs.append((D.cpu().numpy()[:, :N], Dl.cpu().numpy()[:, :N]))
    (Df, Dlf), (Ds, Dls) = outs
    assert np.array_equal(Ds, Ds.T) and np.array_equal(Dls, Dls.T)
    up = np.triu_indices(N)
    assert np.array_equal(Ds[up], Df[up]) and np.array_equal(Dls[up], Dlf[up])
    ref = Zp[:, :N] @ Zp[:, :N].T
    got = Ds.astype(np.float64) + Dls.astype(np.float64)
    assert _rel(got, ref) < 3e-11
