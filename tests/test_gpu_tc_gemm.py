"""The tcgen05 product used by the mixed path, checked on its own through the C ABI.

Operands are FP32 matrices stored exactly as three bf16 pieces; the product of two
such matrices (six piece products, FP32 accumulation) must match the FP64 product
of the same FP32 values to FP32 accuracy.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2mod():
    from paper_1507_02087_gb300 import sp2
    sp2.lib()
    return sp2


def pieces(x32: torch.Tensor) -> torch.Tensor:
    """x = (p0 + p1) + p2 exactly, p_i bf16 (round to nearest even at each step)."""
    p0 = x32.to(torch.bfloat16)
    r1 = x32 - p0.float()
    p1 = r1.to(torch.bfloat16)
    r2 = r1 - p1.float()
    p2 = r2.to(torch.bfloat16)
    assert torch.equal((p0.float() + p1.float()) + p2.float(), x32)
    return torch.stack([p0, p1, p2])


def run(sp2mod, mats, a, b, upper, tile="auto"):
    ld = mats[0].shape[0]
    arena = torch.stack([pieces(m) for m in mats]).contiguous()
    out = torch.full((ld, ld), float("nan"), dtype=torch.float32, device="cuda")
    sp2mod.sp2_test_tc_gemm(arena, ld, len(mats), a, b, upper, out, tile=tile)
    return out


def rel(C, R):
    return float(torch.linalg.norm(C.double() - R) / torch.linalg.norm(R))


@pytest.mark.parametrize("tile", ["128", "pair"])
@pytest.mark.parametrize("ld", [256, 512, 1024, 4096])
def test_general_product(sp2mod, ld, tile):
    g = torch.Generator(device="cpu").manual_seed(ld)
    A = torch.randn(ld, ld, generator=g).float().cuda()
    B = torch.randn(ld, ld, generator=g).float().cuda() * 1e-3
    C = run(sp2mod, [A, B], 0, 1, False, tile)
    R = A.double() @ B.double().T
    assert torch.isfinite(C).all()
    # FP32 accumulation over K = ld terms: relative error a few 1e-6
    assert rel(C, R) < 1e-5
    # each element, against its own magnitude scale (sum of |a_ik b_jk|)
    scale = (A.double().abs() @ B.double().abs().T)
    assert float(((C.double() - R).abs() / scale).max()) < 1e-5


@pytest.mark.parametrize("tile", ["128", "pair"])
@pytest.mark.parametrize("ld", [256, 768, 2048, 4096])
def test_symmetric_square_upper(sp2mod, ld, tile):
    g = torch.Generator(device="cpu").manual_seed(100 + ld)
    X = torch.randn(ld, ld, generator=g, dtype=torch.float64)
    X = ((X + X.T) / (2 * ld ** 0.5)).float().cuda()
    C = run(sp2mod, [X], 0, 0, True, tile)
    R = X.double() @ X.double()
    assert torch.equal(C, C.T)               # mirror writes: exactly symmetric
    assert rel(C, R) < 1e-5


def test_slot_selection_and_zero_border(sp2mod):
    ld = 512
    g = torch.Generator(device="cpu").manual_seed(7)
    mats = [torch.zeros(ld, ld, device="cuda") for _ in range(4)]
    N = 300
    mats[2][:N, :N] = torch.randn(N, N, generator=g).cuda()
    mats[3][:N, :N] = torch.randn(N, N, generator=g).cuda()
    C = run(sp2mod, mats, 2, 3, False)
    R = mats[2].double() @ mats[3].double().T
    assert rel(C, R) < 1e-5
    assert float(C[N:, :].abs().max()) == 0.0 and float(C[:, N:].abs().max()) == 0.0


def test_pair_and_single_tiles_agree(sp2mod):
    # the same six piece products in the same 64-term chunks: both tile kinds give the
    # same FP32 sums up to the tensor cores' internal order within one MMA
    ld = 1536
    g = torch.Generator(device="cpu").manual_seed(5)
    X = torch.randn(ld, ld, generator=g, dtype=torch.float64)
    X = ((X + X.T) / (2 * ld ** 0.5)).float().cuda()
    C1 = run(sp2mod, [X], 0, 0, True, "128")
    C2 = run(sp2mod, [X], 0, 0, True, "pair")
    R = X.double() @ X.double()
    assert rel(C1, R) < 1e-5 and rel(C2, R) < 1e-5
    assert float((C1.double() - C2.double()).abs().max()) < 1e-5 * float(R.abs().max())


def test_tile_argument_checked(sp2mod):
    arena = torch.zeros(1, 3, 384, 384, dtype=torch.bfloat16, device="cuda")
    out = torch.empty(384, 384, device="cuda")
    with pytest.raises(RuntimeError):
        sp2mod.sp2_test_tc_gemm(arena, 384, 1, 0, 0, True, out, tile="pair")   # 384 is not a multiple of 256
    sp2mod.sp2_test_tc_gemm(arena, 384, 1, 0, 0, True, out, tile="auto")       # falls back to 128 x 128 tiles
    assert float(out.abs().max()) == 0.0


# ---- the fp16 piece format (SP2_PREC_FP16X3) ---------------------------------------------------
S16 = 2.0 ** 14


def pieces16(x32: torch.Tensor) -> torch.Tensor:
    """S x = p0 + p1 (+ a remainder below p1's last bit), p_i fp16, S = 2^14."""
    y = x32 * S16
    p0 = y.half()
    p1 = (y - p0.float()).half()
    return torch.stack([p0, p1])


def run16(sp2mod, mats, a, b, upper, tile="auto", lowprec=False):
    ld = mats[0].shape[0]
    arena = torch.stack([pieces16(m) for m in mats]).contiguous()
    out = torch.full((ld, ld), float("nan"), dtype=torch.float32, device="cuda")
    sp2mod.sp2_test_tc_gemm(arena, ld, len(mats), a, b, upper, out, tile=tile, fmt="fp16", lowprec=lowprec)
    return out, arena


def exact16(arena, a, b, lowprec):
    """The format's product of the stored pieces in FP64 (each piece product is exact)."""
    P, Q = arena[a].double(), arena[b].double()
    C = P[0] @ Q[0].T
    if not lowprec:
        C = C + P[0] @ Q[1].T + P[1] @ Q[0].T
    return C / S16 ** 2


@pytest.mark.parametrize("tile", ["128", "pair"])
@pytest.mark.parametrize("ld", [256, 1024, 4096])
@pytest.mark.parametrize("lowprec", [False, True])
def test_fp16_format_product(sp2mod, ld, tile, lowprec):
    g = torch.Generator(device="cpu").manual_seed(300 + ld)
    A = (torch.rand(ld, ld, generator=g) * 2 - 1).float().cuda()
    B = ((torch.rand(ld, ld, generator=g) * 2 - 1) * 1e-2).float().cuda()
    C, arena = run16(sp2mod, [A, B], 0, 1, False, tile, lowprec)
    assert torch.isfinite(C).all()
    R = exact16(arena, 0, 1, lowprec)
    scale = arena[0].double().abs().sum(0) @ arena[1].double().abs().sum(0).T / S16 ** 2
    # the piece products are exact: only the FP32 accumulation (64-term chunks) remains
    assert float(((C.double() - R).abs() / scale).max()) < 1e-5
    # against the FP64 product of the values: 22-bit pieces, three products (2^-21) or one (2^-11)
    E = A.double() @ B.double().T
    assert rel(C, E) < (3e-3 if lowprec else 1e-5)


@pytest.mark.parametrize("tile", ["128", "pair"])
def test_fp16_format_symmetric_square_and_subnormal_pieces(sp2mod, tile):
    # entries down to 1e-9: the low piece of S x is an fp16 subnormal for |x| < 2^-17 and the
    # leading one for |x| < 2^-28; the tensor cores must multiply them exactly, not flush them
    ld = 1024
    g = torch.Generator(device="cpu").manual_seed(11)
    X = torch.randn(ld, ld, generator=g, dtype=torch.float64)
    mag = 10.0 ** torch.empty(ld, ld, dtype=torch.float64).uniform_(-9, -5, generator=g)
    X = (X.sign() * mag)
    X = ((X + X.T) / 2).float().cuda()
    C, arena = run16(sp2mod, [X], 0, 0, True, tile)
    assert torch.equal(C, C.T)
    R = exact16(arena, 0, 0, False)
    scale = arena[0].double().abs().sum(0) @ arena[0].double().abs().sum(0).T / S16 ** 2
    assert float(((C.double() - R).abs() / scale).max()) < 1e-5
    # without the subnormal low pieces the product would be off by about 2^-11 of its scale
    R0 = arena[0][0].double() @ arena[0][0].double().T / S16 ** 2
    assert float(((R0 - R).abs() / scale).max()) > 1e-5


# ---- the tf32 piece format (SP2_PREC_TF32X3) ---------------------------------------------------
def round_tf32(x32: torch.Tensor) -> torch.Tensor:
    """Nearest tf32 value (10 fraction bits), ties away from zero, kept in an FP32 word."""
    b = x32.contiguous().view(torch.int32)
    return ((b + 0x1000) & ~0x1FFF).view(torch.float32)


def pieces32(x32: torch.Tensor) -> torch.Tensor:
    hi = round_tf32(x32)
    lo = round_tf32(x32 - hi)
    return torch.stack([hi, lo])


def run32(sp2mod, mats, a, b, upper, tile="auto", lowprec=False):
    ld = mats[0].shape[0]
    arena = torch.stack([pieces32(m) for m in mats]).contiguous()
    out = torch.full((ld, ld), float("nan"), dtype=torch.float32, device="cuda")
    sp2mod.sp2_test_tc_gemm(arena, ld, len(mats), a, b, upper, out, tile=tile, fmt="tf32", lowprec=lowprec)
    return out, arena


@pytest.mark.parametrize("tile", ["128", "pair"])
@pytest.mark.parametrize("ld", [256, 1024, 4096])
@pytest.mark.parametrize("lowprec", [False, True])
def test_tf32_format_product(sp2mod, ld, tile, lowprec):
    g = torch.Generator(device="cpu").manual_seed(500 + ld)
    A = torch.randn(ld, ld, generator=g).float().cuda()
    B = (torch.randn(ld, ld, generator=g) * 1e-3).float().cuda()
    C, arena = run32(sp2mod, [A, B], 0, 1, False, tile, lowprec)
    assert torch.isfinite(C).all()
    P, Q = arena[0].double(), arena[1].double()
    R = P[0] @ Q[0].T if lowprec else P[0] @ Q[0].T + P[0] @ Q[1].T + P[1] @ Q[0].T
    scale = P.abs().sum(0) @ Q.abs().sum(0).T
    # each piece product is exact (tf32 x tf32 fits FP32); only the FP32 accumulation remains
    assert float(((C.double() - R).abs() / scale).max()) < 1e-5
    E = A.double() @ B.double().T
    assert rel(C, E) < (3e-3 if lowprec else 1e-5)


@pytest.mark.parametrize("tile", ["128", "pair"])
def test_tf32_format_symmetric_square(sp2mod, tile):
    ld = 1536 if tile == "128" else 1792
    g = torch.Generator(device="cpu").manual_seed(21)
    X = torch.randn(ld, ld, generator=g, dtype=torch.float64)
    X = ((X + X.T) / (2 * ld ** 0.5)).float().cuda()
    C, arena = run32(sp2mod, [X], 0, 0, True, tile)
    assert torch.equal(C, C.T)
    assert rel(C, X.double() @ X.double()) < 1e-5
