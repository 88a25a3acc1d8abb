"""The tensor-core kernel's bounded waits, made to run out without any GPU fault.

A testing entry point launches the 128 x 128 (one SM per tile) product with every mbarrier
wait limited to 50 ms and CTA 0 leaving the first stage of its copy ring unarmed.  Its MMA
thread's wait must give up, the kernel must report SP2_ERR_TIMEOUT and return (the CTA's
other warps give up too, wait for the copies they issued and free their tensor memory),
the other CTAs must finish their tiles, and the context must stay usable: a fresh product
and a fresh purification afterwards are green.
"""
import numpy as np
import pytest
import torch

from oracle import sp2_oracle as o
from paper_1507_02087_gb300 import inputs

pytestmark = pytest.mark.gpu


def pieces(x32):
    p0 = x32.to(torch.bfloat16)
    r1 = x32 - p0.float()
    p1 = r1.to(torch.bfloat16)
    p2 = (r1 - p1.float()).to(torch.bfloat16)
    return torch.stack([p0, p1, p2])


def test_bounded_wait_gives_up_and_context_stays_usable():
    from paper_1507_02087_gb300 import sp2
    L = sp2.lib()
    ld = 1024                                 # 64 tiles of 128 x 128, one per CTA
    g = torch.Generator(device="cpu").manual_seed(3)
    X = torch.randn(ld, ld, generator=g).float().cuda()
    arena = pieces(X).unsqueeze(0).contiguous()
    out = torch.full((ld, ld), float("nan"), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    rc = L.sp2_test_tc_timeout(arena.data_ptr(), ld, 50, out.data_ptr(), s)
    assert rc == 4                            # SP2_ERR_TIMEOUT
    R = X.double() @ X.double().T
    done = torch.ones(ld, ld, dtype=torch.bool, device="cuda")
    done[:128, :128] = False                  # CTA 0's tile (0, 0) is abandoned
    err = (out.double() - R).abs() / (X.double().abs() @ X.double().abs().T)
    assert float(err[done].max()) < 1e-5      # every other CTA finished its tile
    assert L.sp2_test_tc_timeout(arena.data_ptr(), ld, 0, out.data_ptr(), s) == 1    # limit checked
    # the context is still usable: the same product without the hook, then a purification
    out2 = torch.empty_like(out)
    sp2.sp2_test_tc_gemm(arena, ld, 1, 0, 0, False, out2, tile="128")
    assert float(((out2.double() - R).abs() / (X.double().abs() @ X.double().abs().T)).max()) < 1e-5
    case = inputs.dense_gapped(300, 140, gap=0.05, seed=9)
    with sp2.Purifier(300, 140, "mixed", tile="128") as P:
        D = P.run(case.F.cuda()).cpu().numpy()
        info = P.info()
    assert info["status"] == 0
    assert o.rel_error(D, o.sp2(case.F.numpy(), 140).D, 140) <= 1e-6
