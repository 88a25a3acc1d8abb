"""Block-sparse path (32 x 32 FP32 blocks, Frobenius block truncation) through the C ABI.

Index work (the truncation decision and the symbolic square) must equal the host's bit
for bit given the same stored blocks.

The purification is compared with two oracles that apply the same truncation after every
step (Alg. 1, X~_i = X_i + E_i): the FP64 one, and the one that also rounds every stored
iterate to FP32 (E_i = storage rounding + truncation), which is what the GPU stores.  The
block products run on the tensor cores by default (two fp16 pieces of 2^14 x per block,
three piece products, FP32 accumulation in chunks): the stop must be within one square of
the FP32-storage oracle's.

D tolerance, derived (not measured): one square's products carry a relative error of at
most about 2^-20 of ||X||_F (three 22-bit piece products, FP32 chunk sums); the errors of
the n squares are independent, so they add like sqrt(n), and a perturbation of the iterate
moves the occupied subspace by at most its size over the scaled gap g0 of X_0 (the gap only
widens under the SP2 maps); ||X||_F <= sqrt(nocc) for a projector-like iterate.  Hence
||D - D_ref||_F / sqrt(nocc) <= sqrt(n) 2^-20 / g0, with g0 ~ 0.31 on these lattices
(about 1.2e-5 at n = 15; measured: 4e-7).

The FP32 CUDA-core block products (an option) accumulate every element in one sequential
FP32 chain over all N terms: tiny terms that follow the large diagonal term are lost, which
biases the trace at the rounding floor and lets the trace-chosen polynomial repeat there
(§4.2: such runs are not bounded under trace selection) for up to four squares before the
order test can fire; a CPU emulation of that exact arithmetic reproduces its histories digit
for digit.  Its stop is checked in that wider window.
"""
import math

import numpy as np
import pytest
import torch

from oracle import bsr_oracle as bo
from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu


def d_tol(n, F, nocc):
    """sqrt(n) 2^-20 / g0, g0 = the scaled gap of X_0 (module notes)."""
    lmin, lmax = o.gershgorin_bounds(F)
    lam = np.linalg.eigvalsh(F)
    g0 = (lam[nocc] - lam[nocc - 1]) / (lmax - lmin)
    return math.sqrt(max(n, 1)) * 2.0 ** -20 / g0


def assert_parity(info, D, F, nocc, tau, **kw):
    """Stop within one square of the FP32-storage oracle; D within the derived tolerance of the
    FP64 oracle (and of the FP32-storage one)."""
    ref = bo.sp2_bsr(F, nocc, 32, tau, **kw)
    ref32 = bo.sp2_bsr(F, nocc, 32, tau, storage="fp32", **kw)
    assert abs(info["n_iter"] - ref32.n) <= 1, (info["n_iter"], ref32.n)
    tol = d_tol(info["n_iter"], F, nocc)
    assert o.rel_error(D, ref.D, nocc) <= tol
    assert o.rel_error(D, ref32.D, nocc) <= tol
    return ref


@pytest.fixture(scope="module")
def sp2mod():
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    return sp2


def test_truncation_decision_bit_exact(sp2mod):
    g = np.random.Generator(np.random.PCG64(5))
    nb, b = 24, 32
    N = nb * b
    tau = 1e-4
    X = g.standard_normal((N, N)) * 1e-3
    # blocks spread around the threshold: scale each block so its norm is tau * f
    for I in range(nb):
        for J in range(nb):
            f = g.choice([0.5, 0.999999, 1.0, 1.000001, 2.0, 30.0])
            blk = X[I * b:(I + 1) * b, J * b:(J + 1) * b]
            blk *= tau * f / np.linalg.norm(blk)
    X32 = X.astype(np.float32)
    keep_gpu = torch.zeros(nb * nb, dtype=torch.uint8, device="cuda")
    rc = sp2mod.lib().sp2_test_bsr_keep(torch.from_numpy(X32).cuda().data_ptr(), N, tau, 0, keep_gpu.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    keep_ref = bo.keep_mask(X32.astype(np.float64), b, tau)
    assert np.array_equal(keep_gpu.cpu().numpy().reshape(nb, nb).astype(bool), keep_ref)
    assert 0 < keep_ref.sum() < nb * nb


def _keep_gpu(sp2mod, X32, tau, rule):
    N = X32.shape[0]
    nb = N // 32
    keep = torch.zeros(nb * nb, dtype=torch.uint8, device="cuda")
    rc = sp2mod.lib().sp2_test_bsr_keep(torch.from_numpy(np.ascontiguousarray(X32)).cuda().data_ptr(), N, tau,
                                        rule, keep.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    return keep.cpu().numpy().reshape(nb, nb).astype(bool)


def _spread_blocks(nb, seed):
    """Symmetric block matrix with block norms spread over many decades, exact ties (one
    block repeated), zero blocks and identity-dominated diagonal blocks; FP32 values."""
    g = np.random.Generator(np.random.PCG64(seed))
    b = 32
    X = np.zeros((nb * b, nb * b))
    proto = g.standard_normal((b, b))
    for I in range(nb):
        for J in range(I, nb):
            kind = g.integers(0, 4)
            if kind == 0:
                blk = g.standard_normal((b, b)) * 10.0 ** g.uniform(-9, 0)
            elif kind == 1:
                blk = proto * 1e-5                       # the same block many times: exact ties
            elif kind == 2:
                blk = np.zeros((b, b))
            else:
                blk = g.standard_normal((b, b)) * 1e-4
            if I == J:
                blk = 0.5 * (blk + blk.T) + np.eye(b)
            X[I * b:(I + 1) * b, J * b:(J + 1) * b] = blk
            X[J * b:(J + 1) * b, I * b:(I + 1) * b] = blk.T
    return X.astype(np.float32), proto


@pytest.mark.parametrize("nb,seed", [(3, 1), (24, 2), (90, 3)])
def test_error_truncation_decision_bit_exact(sp2mod, nb, seed):
    # budgets that cut inside a tie group among them
    b = 32
    X32, proto = _spread_blocks(nb, seed)
    n2 = bo.block_norms2(X32.astype(np.float64), b)
    tie = float(np.float64(np.linalg.norm((proto * 1e-5).astype(np.float32).astype(np.float64)) ** 2))
    for tau in (0.0, 1e-7, 1e-4, 3e-3, np.sqrt(7.5 * tie), 1e3):
        keep_gpu = _keep_gpu(sp2mod, X32, tau, 1)
        keep_ref = bo.keep_mask_error(X32.astype(np.float64), b, tau)
        assert np.array_equal(keep_gpu, keep_ref), tau
        E = X32.astype(np.float64) * np.kron(~keep_ref, np.ones((b, b)))
        assert np.linalg.norm(E) <= tau * (1 + 1e-9) + 1e-300
    assert n2.size == nb * nb


@pytest.mark.parametrize("nb,seed", [(3, 1), (24, 2), (90, 3)])
def test_mixed_truncation_decision_bit_exact(sp2mod, nb, seed):
    # rule 2 against the oracle's sequential walk; tau = 2.5 x the tied norm lets each block
    # row take two of the tied blocks, so the cut falls inside the tie group
    b = 32
    X32, proto = _spread_blocks(nb, seed)
    tie = float(np.linalg.norm((proto * 1e-5).astype(np.float32).astype(np.float64)))
    for tau in (0.0, 1e-7, 1e-4, 3e-3, 2.5 * tie, 1e3):
        keep_gpu = _keep_gpu(sp2mod, X32, tau, 2)
        keep_ref = bo.keep_mask_mixed(X32.astype(np.float64), b, tau)
        assert np.array_equal(keep_gpu, keep_ref), tau
        E = X32.astype(np.float64) * np.kron(~keep_ref, np.ones((b, b)))
        M = np.sqrt(bo.block_norms2(E, b))
        assert M.sum(axis=1).max() <= tau * (1 + 1e-9) + 1e-300
        assert np.linalg.norm(M, 2) <= tau * (1 + 1e-9) + 1e-300


@pytest.mark.parametrize("dims,tau", [((32, 8, 4), 1e-4), ((32, 8, 8), 1e-5)])
def test_bsr_mixed_rule_and_mixed_norm_stop(sp2mod, dims, tau):
    # the §6 pairing: mixed-norm truncation and the mixed-norm stop with the 32 x 32 blocks
    tb, (rp, ci, vals) = tb_case(dims)
    F = tb.dense().numpy()
    with sp2mod.BsrPurifier(tb.N, tb.nocc, tau, rule="mixed", norm="mixed") as P:
        D = P.run(rp, ci, vals)
        info = P.info()
    assert info["status"] == 0
    assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    ref = assert_parity(info, D.cpu().numpy(), F, tb.nocc, tau, rule="mixed", norm="mixed")
    Dn = D.cpu().numpy()
    assert np.array_equal(Dn, Dn.T)
    # the recorded measure is m_i (Lanczos on the block-norm matrix, exact for nb <= 32 steps),
    # equal to the oracle's on the first iterates before FP32 and FP64 iterates drift apart
    for i in range(3):
        assert info["v"][i] == pytest.approx(ref.v[i], rel=1e-4)
    with sp2mod.BsrPurifier(tb.N, tb.nocc, tau, rule="mixed") as P:
        P.run(rp, ci, vals)
        fro = P.info()
    for i in range(min(3, fro["hist_len"])):
        assert info["v"][i] <= fro["v"][i] * (1 + 1e-6)


def test_bsr_norm_options(sp2mod):
    tb, (rp, ci, vals) = tb_case((32, 2, 2))
    with pytest.raises(sp2mod.SP2Error):
        sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-4, norm="spectral")


@pytest.mark.parametrize("dims,tau", [((32, 8, 4), 1e-6), ((32, 8, 8), 1e-4)])
def test_bsr_error_rule_against_oracle(sp2mod, dims, tau):
    tb, (rp, ci, vals) = tb_case(dims)
    F = tb.dense().numpy()
    with sp2mod.BsrPurifier(tb.N, tb.nocc, tau, rule="error") as P:
        D = P.run(rp, ci, vals)
        info = P.info()
    assert info["status"] == 0
    assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert_parity(info, D.cpu().numpy(), F, tb.nocc, tau, rule="error")
    Dn = D.cpu().numpy()
    assert np.array_equal(Dn, Dn.T)


@pytest.mark.parametrize("nb,density", [(1, 1.0), (5, 0.4), (70, 0.08), (130, 0.03)])
def test_symbolic_square_bit_exact(sp2mod, nb, density):
    g = np.random.Generator(np.random.PCG64(nb))
    m = g.random((nb, nb)) < density
    m = m | m.T
    np.fill_diagonal(m, True)
    out = np.zeros((nb, nb), dtype=np.uint8)
    mask = np.ascontiguousarray(m.astype(np.uint8))
    rc = sp2mod.lib().sp2_test_bsr_square_pattern(mask.ctypes.data, nb, out.ctypes.data)
    assert rc == 0
    ref = np.triu(bo.square_pattern(m))
    assert np.array_equal(out.astype(bool), ref)


def tb_case(dims):
    tb = inputs.tight_binding(dims=dims)
    rp, ci, vals = tb.bsr(32)
    return tb, (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(vals).cuda())


@pytest.mark.parametrize("dims,tau", [((32, 8, 4), 0.0), ((32, 8, 8), 1e-6), ((32, 16, 8), 1e-4)])
def test_bsr_sp2_against_oracle(sp2mod, dims, tau):
    tb, (rp, ci, vals) = tb_case(dims)
    F = tb.dense().numpy()
    with sp2mod.BsrPurifier(tb.N, tb.nocc, tau) as P:
        D = P.run(rp, ci, vals)
        info = P.info()
    assert info["status"] == 0
    assert info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    ref = assert_parity(info, D.cpu().numpy(), F, tb.nocc, tau)
    assert info["lambda_min"] == pytest.approx(ref.lmin, rel=1e-12)
    assert info["lambda_max"] == pytest.approx(ref.lmax, rel=1e-12)
    Dn = D.cpu().numpy()
    assert np.array_equal(Dn, Dn.T)
    # the stored pattern of D is what the truncation keeps
    assert info["nnzb"] == int(np.count_nonzero(np.abs(Dn).reshape(tb.N // 32, 32, tb.N // 32, 32).sum(axis=(1, 3))))


def test_bsr_launch_modes_agree_and_errors(sp2mod):
    tb, (rp, ci, vals) = tb_case((32, 8, 4))
    out = []
    for mode in (0, 1):
        with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-5, launch_mode=mode) as P:
            out.append((P.run(rp, ci, vals), P.info()["n_iter"]))
    assert out[0][1] == out[1][1] and torch.equal(out[0][0], out[1][0])
    bad = vals.clone()
    bad[0, 1, 2] = float("nan")
    with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-5) as P:
        D = P.run(rp, ci, bad)
        assert P.info()["status"] == 3 and bool(torch.isnan(D).all())


def test_bsr_launch_modes_agree_mixed_rule_stop_and_acc(sp2mod):
    # the mixed-norm selection, the Lanczos mixed-norm stop and SP2-ACC, in the graph and as
    # plain stream launches: the same kernels, so the same bits and the same recorded m_i
    tb, (rp, ci, vals) = tb_case((32, 8, 4))
    lam = np.linalg.eigvalsh(tb.dense().numpy())
    homo, lumo = float(lam[tb.nocc - 1]), float(lam[tb.nocc])
    for acc in (None, (homo - 1e-2, homo, lumo, lumo + 1e-2)):
        out = []
        for mode in (0, 1):
            with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-4, launch_mode=mode, rule="mixed", norm="mixed") as P:
                if acc is not None:
                    P.set_homo_lumo(acc)
                D = P.run(rp, ci, vals)
                out.append((D, P.info()))
        (D0, i0), (D1, i1) = out
        assert i0["status"] == 0 and i0["n_iter"] == i1["n_iter"] and torch.equal(D0, D1)
        assert list(i0["v"]) == list(i1["v"]) and i0["nnzb"] == i1["nnzb"]


@pytest.mark.parametrize("rule,norm", [("error", "fro"), ("mixed", "mixed")])
def test_bsr_full_size_32cubed_a_posteriori(sp2mod, rule, norm):
    """The 32^3 lattice (N = 32768) in the benchmark's configuration (error-controlled rule,
    tau = 1e-4, graph launch).  No oracle runs at this size, so the test checks what holds at any
    size and bounds the distance to the exact projector P from it: with P~ the projector onto
    the eigenvectors of D above 1/2, ||D - P~||_F <= ||D^2 - D||_F / (1 - 2 m) (m the largest
    distance of an eigenvalue of D from {0, 1}) and, by the sin-theta theorem with the gap delta
    of F, ||P~ - P||_F <= ||[F, P~]||_F / delta <= (||[F, D]||_F + 2 ||F||_2 ||D - P~||_F) / delta."""
    import math
    tb = inputs.tight_binding(L=32)
    rp, ci, vals = tb.bsr(32)
    rp_d, ci_d, vals_d = (torch.from_numpy(x).cuda() for x in (rp, ci, vals))
    with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-4, rule=rule, norm=norm) as P:
        D = P.run(rp_d, ci_d, vals_d)
        info = P.info()
    assert info["status"] == 0 and info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    assert torch.equal(D, D.T)
    nocc = tb.nocc
    tr = float(torch.trace(D))
    # F D from the sparse F in FP64 (onsite diagonal, hopping -t to the six neighbours)
    r = torch.from_numpy(tb.rows).cuda()
    c = torch.from_numpy(tb.cols).cuda()
    idx = torch.cat([torch.stack([r, c]), torch.arange(tb.N, device="cuda").repeat(2, 1)], dim=1)
    val = torch.cat([torch.full((r.numel(),), -tb.hop, dtype=torch.float64, device="cuda"),
                     torch.from_numpy(tb.onsite).cuda()])
    Fs = torch.sparse_coo_tensor(idx, val, (tb.N, tb.N)).coalesce()
    FD = torch.sparse.mm(Fs, D)
    comm = float(torch.linalg.norm(FD - FD.T))            # [F, D] = F D - (F D)^T for symmetric F, D
    del FD
    # D^2 - D with FP32 products (no TF32): error ~1e-7 of ||D||_F^2 / sqrt(N), far below the FP32 floor of D
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    D32 = D.float()
    idem = float(torch.linalg.norm((D32 @ D32).double() - D))
    torch.backends.cuda.matmul.allow_tf32 = prev
    del D32
    # the gap: without disorder the bands are +-sqrt(Delta^2 + eps_k^2) (bipartite lattice), so
    # |lambda| >= Delta = 1; the onsite disorder moves every eigenvalue by at most its largest
    # magnitude (Weyl), so the gap around 0 is at least 2 (Delta - max |noise|)
    onsite = tb.onsite
    delta_gap = 2.0 * (1.0 - float(np.max(np.abs(np.abs(onsite) - 1.0))))
    Fnorm = float(np.max(np.abs(onsite))) + 6 * tb.hop     # Gershgorin
    m = 0.01                                               # eigenvalues of D within 0.01 of {0, 1}:
    assert idem < m / 2                                    # |d - d^2| >= m (1 - m) > m / 2 otherwise
    d_ptilde = idem / (1 - 2 * m)
    bound = d_ptilde + (comm + 2 * Fnorm * d_ptilde) / delta_gap
    print(f"trace err {tr - nocc:.3e} idem {idem:.3e} comm {comm:.3e} gap {delta_gap:.3f} "
          f"bound/sqrt(nocc) {bound / math.sqrt(nocc):.3e} n {info['n_iter']} kept {info['nnzb']}")
    assert abs(tr - nocc) < 0.5                            # P~ has rank nocc
    # budget: n truncations of ||E_i||_F <= tau, each moving the subspace by at most
    # tau (1 + 2 ||F|| / delta) / delta to first order: 15 * 1e-4 * 3.7 / 1.6 / 128 ~ 3e-5 per
    # sqrt(nocc), plus the FP32 floor of the stored blocks (measured bound: 8e-6)
    budget = info["n_iter"] * 1e-4 * (1 + 2 * Fnorm / delta_gap) / delta_gap / math.sqrt(nocc)
    if rule == "error":
        assert bound / math.sqrt(nocc) <= budget + 1e-5
    else:
        # ||E_i||_2 <= tau but ||E_i||_F up to sqrt(N) tau: a looser Frobenius budget
        assert bound / math.sqrt(nocc) <= 1e-3


@pytest.mark.parametrize("rule,norm", [("error", "fro"), ("mixed", "mixed")])
def test_bsr_acc_against_oracle(sp2mod, rule, norm):
    # SP2-ACC (Alg. 4 / Alg. 5) with the block truncation: the schedule comes from the run's
    # Gershgorin bounds, so with the same bounds the oracle's polynomial sequence must agree
    tb, (rp, ci, vals) = tb_case((32, 8, 4))
    F = tb.dense().numpy()
    lam = np.linalg.eigvalsh(F)
    homo, lumo = float(lam[tb.nocc - 1]), float(lam[tb.nocc])
    acc = (homo - 1e-2, homo, lumo, lumo + 1e-2)
    with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-4, rule=rule, norm=norm) as P:
        D0 = P.run(rp, ci, vals)
        i0 = P.info()
        P.set_homo_lumo(acc)
        D = P.run(rp, ci, vals).cpu().numpy()
        info = P.info()
        with pytest.raises(sp2mod.SP2Error):
            P.set_homo_lumo((0.1, 0.0, 0.2, 0.3))
        P.set_homo_lumo(None)
        D1 = P.run(rp, ci, vals)
        i1 = P.info()
    assert info["status"] == 0
    ref = assert_parity(info, D, F, tb.nocc, 1e-4, rule=rule, norm=norm, acc=acc,
                        bounds=(info["lambda_min"], info["lambda_max"]))
    m = min(info["n_iter"], ref.n)
    assert list(info["p"][1:m + 1]) == ref.p[1:m + 1]
    assert info["n_iter"] < i0["n_iter"]
    assert i1["n_iter"] == i0["n_iter"] and torch.equal(D0, D1)       # back to Alg. 3, same bits


def test_bsr_caller_bounds(sp2mod):
    # outer bounds from Weyl's inequality in place of Gershgorin's: without disorder the extreme
    # eigenvalues are +-sqrt(delta^2 + (6t)^2) (k = 0 is on every periodic lattice), and the onsite
    # disorder moves each eigenvalue by at most its largest magnitude
    tb, (rp, ci, vals) = tb_case((32, 8, 4))
    F = tb.dense().numpy()
    mn = float(np.max(np.abs(np.abs(tb.onsite) - 1.0)))
    e = float(np.sqrt(1.0 + (6 * tb.hop) ** 2)) + mn
    bounds = (-e, e)
    lam = np.linalg.eigvalsh(F)
    assert bounds[0] <= lam[0] and lam[-1] <= bounds[1]
    with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-5, rule="error") as P:
        P.run(rp, ci, vals)
        n_gersh = P.info()["n_iter"]
        P.set_bounds(bounds)
        D = P.run(rp, ci, vals).cpu().numpy()
        info = P.info()
        with pytest.raises(sp2mod.SP2Error):
            P.set_bounds((1.0, 1.0))
        P.set_bounds(None)
        P.run(rp, ci, vals)
        assert P.info()["n_iter"] == n_gersh
    assert (info["lambda_min"], info["lambda_max"]) == bounds
    assert info["status"] == 0 and info["n_iter"] <= n_gersh
    assert_parity(info, D, F, tb.nocc, 1e-5, rule="error", bounds=bounds)


@pytest.mark.parametrize("dims,tau,rule", [((32, 8, 4), 1e-6, "error"), ((32, 8, 8), 1e-4, "error"),
                                           ((32, 8, 8), 1e-6, "block")])
def test_bsr_cuda_core_products_option(sp2mod, dims, tau, rule):
    # the FP32 CUDA-core block products: same index work and truncation, D within the derived
    # tolerance; the stop in the window of its sequential sums (module notes)
    tb, (rp, ci, vals) = tb_case(dims)
    F = tb.dense().numpy()
    with sp2mod.BsrPurifier(tb.N, tb.nocc, tau, rule=rule, products="cuda") as P:
        D = P.run(rp, ci, vals).cpu().numpy()
        info = P.info()
    assert info["status"] == 0 and info["stop_reason"] in (o.STOP_ORDER, o.STOP_TRACE_GUARD)
    ref = bo.sp2_bsr(F, tb.nocc, 32, tau, rule=rule)
    ref32 = bo.sp2_bsr(F, tb.nocc, 32, tau, rule=rule, storage="fp32")
    assert ref32.n - 1 <= info["n_iter"] <= ref32.n + 4
    assert o.rel_error(D, ref.D, tb.nocc) <= d_tol(info["n_iter"], F, tb.nocc)
    assert np.array_equal(D, D.T)


def test_bsr_tensor_core_products_deterministic(sp2mod):
    # the same input twice, and the graph against stream launches: the same bits
    tb, (rp, ci, vals) = tb_case((32, 8, 8))
    out = []
    for mode in (0, 0, 1):
        with sp2mod.BsrPurifier(tb.N, tb.nocc, 1e-4, rule="error", launch_mode=mode) as P:
            out.append((P.run(rp, ci, vals), P.info()))
    for D, info in out[1:]:
        assert info["n_iter"] == out[0][1]["n_iter"] and torch.equal(D, out[0][0])
    assert out[0][1]["status"] == 0
