"""The warm-start network's matrix products on both engines (tcgen05 tensor-core tiles
and warp-level mma.sync tiles), called through the C ABI on device buffers, against an
FP64 product of the same BF16 operands:

* C = A B^T (+ bias) (relu) within the FP32 accumulation bound
  |C - C_64| <= 2^-22 K (|A| |B|^T + |bias|) elementwise (K terms, each rounding once);
* the BF16 copy is the round-to-nearest-even BF16 of the FP32 result, bit for bit;
* ragged shapes: M not a multiple of the 128-row tile (tcgen05), K not a multiple of its
  64-wide chunk, N split into several tiles, N of a single 16-wide tile;
* the two engines agree within twice that bound; no wait gives up (err stays 0).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SHAPES = [(200, 256, 16), (256, 256, 512), (16, 16, 256), (1000, 512, 80), (128, 48, 64), (33, 256, 272),
          (4096, 256, 256)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()


def _run(od, A, B, bias, M, N, K, relu, engine):
    C = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    Cb = torch.zeros((M, N), device="cuda", dtype=torch.bfloat16)
    err = torch.zeros(1, device="cuda", dtype=torch.int32)
    od.od_gemm_bf16(A.data_ptr(), B.data_ptr(), bias.data_ptr() if bias is not None else 0, C.data_ptr(),
                    Cb.data_ptr(), M, N, K, relu, engine, err.data_ptr())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return C, Cb


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("relu", [0, 1])
def test_products_match_fp64(M, N, K, relu):
    import paper_2205_06557_gb300 as od

    torch.cuda.set_device(0)
    g = torch.Generator(device="cpu").manual_seed(M * 7919 + N * 31 + K + relu)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = (torch.randn(N, K, generator=g) / np.sqrt(K)).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).cuda() if relu else None
    a64, b64 = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = a64 @ b64.T
    mag = np.abs(a64) @ np.abs(b64).T
    if bias is not None:
        ref = ref + bias.double().cpu().numpy()[None, :]
        mag = mag + np.abs(bias.double().cpu().numpy())[None, :]
    if relu:
        ref = np.maximum(ref, 0.0)
    bound = 2.0 ** -22 * K * mag + 1e-30
    out = {}
    for engine in (od.GEMM_TCGEN05, od.GEMM_MMA_SYNC):
        if engine == od.GEMM_MMA_SYNC and M % 16:
            continue
        C, Cb = _run(od, A, B, bias, M, N, K, relu, engine)
        c = C.double().cpu().numpy()
        assert np.isfinite(c).all()
        excess = np.abs(c - ref) / bound
        assert excess.max() <= 1.0, (engine, float(excess.max()))
        assert torch.equal(Cb.cpu().view(torch.int16), C.to(torch.bfloat16).cpu().view(torch.int16))
        out[engine] = c
    if len(out) == 2:
        assert (np.abs(out[0] - out[1]) / bound).max() <= 2.0


def test_bad_sizes_are_rejected():
    import paper_2205_06557_gb300 as od

    A = torch.zeros(32, 32, device="cuda", dtype=torch.bfloat16)
    C = torch.zeros(32, 32, device="cuda")
    err = torch.zeros(1, device="cuda", dtype=torch.int32)
    for M, N, K, engine in [(32, 24, 32, 0), (32, 32, 24, 0), (24, 32, 32, 1), (32, 32, 32, 2), (0, 32, 32, 0)]:
        with pytest.raises(od.OdError):
            od.od_gemm_bf16(A.data_ptr(), A.data_ptr(), 0, C.data_ptr(), 0, M, N, K, 0, engine, err.data_ptr())
