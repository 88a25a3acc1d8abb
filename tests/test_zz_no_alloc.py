"""The allocation-free FP64 entry point, for callers that cannot call cudaMalloc
(for example code that runs under another component's device allocator, or inside a
loop where entering the allocator is not allowed).  It keeps its workspace in one
fixed device array inside the library instead of allocating.

Checked through the C ABI on consecutive calls that share the same workspace, the
largest allowed size included: against the regular FP64 entry point (sp2_run with an
SP2_PREC_FP64 handle and default options), which runs the same kernels with the same
options, so the results must be identical bit for bit; and against the CPU FP64 oracle,
within the FP64 tolerance the other tests use (1e-10, stop within one iteration), so
that a fault shared by both GPU entry points is caught too.  This file is collected last
so that a run that stops at the first failure has already run every other test.
"""
import pytest
import torch

from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-10


def noalloc(sp2mod, F, nocc):
    N = F.shape[0]
    D = torch.full_like(F, float("nan"))
    info = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = sp2mod.lib().sp2_run_fp64_noalloc(F.data_ptr(), D.data_ptr(), N, nocc, info.data_ptr(), stream)
    assert rc == 0
    torch.cuda.synchronize()
    return D, info.cpu().tolist()


def regular(sp2mod, F, nocc):
    with sp2mod.Purifier(F.shape[0], nocc, "fp64") as P:
        D = P.run(F)
        info = P.info()
    return D, info


def test_noalloc_matches_regular_entry_and_oracle_on_consecutive_calls():
    from oracle import sp2_oracle as o
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    # the largest allowed size first, then smaller ones: each later call reuses the
    # workspace the earlier ones filled, including the region beyond its own padded size
    for N, nocc, gap, seed in [(512, 250, 0.05, 20), (500, 240, 0.05, 21), (200, 90, 0.1, 22)]:
        case = inputs.dense_gapped(N, nocc, gap=gap, seed=seed)
        F = case.F.cuda()
        Dn, info_n = noalloc(sp2, F, nocc)
        Dr, info_r = regular(sp2, F, nocc)
        assert info_n[0] == 0
        assert info_n[1] == info_r["n_iter"] and info_n[3] == info_r["hist_len"]
        assert torch.equal(Dn, Dr)
        ref = o.sp2(case.F.numpy(), nocc)
        assert abs(info_n[1] - ref.n) <= 1
        assert o.rel_error(Dn.cpu().numpy(), ref.D, nocc) <= TOL_FP64


def test_noalloc_rejects_oversize_and_bad_arguments():
    from paper_1507_02087_gb300 import sp2
    L = sp2.lib()
    F = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    D = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert L.sp2_run_fp64_noalloc(F.data_ptr(), D.data_ptr(), 513, 10, None, s) == 1
    assert L.sp2_run_fp64_noalloc(F.data_ptr(), D.data_ptr(), 4, 5, None, s) == 1
    assert L.sp2_run_fp64_noalloc(None, D.data_ptr(), 4, 2, None, s) == 1
    assert L.sp2_run_fp64_noalloc(F.data_ptr(), F.data_ptr(), 4, 2, None, s) == 1
