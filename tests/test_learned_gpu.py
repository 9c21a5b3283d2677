"""Learned coarse-grid corrector on the GPU: the tcgen05 convolution (forward,
last layer, input gradient with ReLU mask), the weight-gradient reduction and
the restriction against the FP64 oracle, then the corrected step and
training.

Bars: convolution outputs are BF16, so they are compared with the oracle on
the same BF16-rounded inputs and weights within 1e-2 relative (BF16 has an
8-bit mantissa; the accumulation is FP32); FP32 outputs within 1e-4.

Two shapes: SMALL gives each CTA of the persistent convolution one block;
MULTI (64 x 128 x 128 points, 2048 blocks of 8 x 16 x 4 on at most 148 CTAs)
gives every CTA six or more blocks, so the reuse of both shared-memory stages, both TMEM
accumulator buffers and every mbarrier phase after the first are compared
with the oracle too."""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu

SMALL = (8, 16, 64)   # (nz, ny, nx): nx a multiple of 64 (weight gradient), nz of 8, ny of 16
MULTI = (64, 128, 128)
SHAPES = pytest.mark.parametrize("shape", [SMALL, MULTI], ids=["small", "multi"])


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def rand_act(seed, ci, shape, scale=1.0):
    g = np.random.default_rng(seed)
    x = np.zeros(shape + (16,), dtype=np.float32)
    x[..., :ci] = g.normal(size=shape + (ci,)) * scale
    return bf16_round(x)


def to_dev_bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16).contiguous()


def close(gpu, ref, rtol):
    scale = max(1e-6, float(np.max(np.abs(ref))))
    err = float(np.max(np.abs(gpu - ref)))
    assert err <= rtol * scale, (err, scale)


@SHAPES
@pytest.mark.parametrize("ci,co", [(16, 16), (3, 16)])
def test_conv_forward_relu(ci, co, shape):
    x = rand_act(1, ci, shape)
    g = np.random.default_rng(2)
    W = bf16_round(g.normal(size=(27, ci, co)) * 0.2)
    b = g.normal(size=(co,)).astype(np.float32) * 0.1
    out, st = ls.conv3_bf16(to_dev_bf16(x), torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), 0)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oracle.relu(oracle.conv3_fwd(x[..., :ci].astype(np.float64), W, b))
    close(out.float().cpu().numpy()[..., :co], ref, 1e-2)


@SHAPES
def test_conv_last_layer_fp32(shape):
    x = rand_act(3, 16, shape)
    g = np.random.default_rng(4)
    W = bf16_round(g.normal(size=(27, 16, 1)) * 0.2)
    b = np.array([0.3], dtype=np.float32)
    out, st = ls.conv3_bf16(to_dev_bf16(x), torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), 1)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oracle.conv3_fwd(x.astype(np.float64), W, b)[..., 0]
    close(out.cpu().numpy(), ref, 1e-4)


@SHAPES
@pytest.mark.parametrize("ci,co", [(16, 16), (16, 1)])
def test_conv_input_gradient_masked(ci, co, shape):
    """mode 2: conv^T of the output gradient, times the ReLU mask."""
    gy = np.zeros(shape + (16,), dtype=np.float32)
    gy[..., :co] = np.random.default_rng(5).normal(size=shape + (co,))
    gy = bf16_round(gy)
    g = np.random.default_rng(6)
    W = bf16_round(g.normal(size=(27, ci, co)) * 0.2)
    mask = bf16_round(np.maximum(g.normal(size=shape + (16,)), 0))
    out, st = ls.conv3_bf16(to_dev_bf16(gy), torch.from_numpy(W).cuda(), None, 2, mask=to_dev_bf16(mask))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oracle.conv3_bwd_data(gy[..., :co].astype(np.float64), W) * (mask[..., :ci] > 0)
    close(out.float().cpu().numpy()[..., :ci], ref, 1e-2)


@SHAPES
@pytest.mark.parametrize("ci,co", [(16, 16), (3, 16), (16, 1)])
def test_weight_gradient(ci, co, shape):
    x = rand_act(7, ci, shape)
    gy = np.zeros(shape + (16,), dtype=np.float32)
    gy[..., :co] = np.random.default_rng(8).normal(size=shape + (co,))
    gy = bf16_round(gy)
    dW, db, st = ls.conv3_wgrad(to_dev_bf16(x), to_dev_bf16(gy), ci, co, with_status=True)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rW, rb = oracle.conv3_bwd_weight(x[..., :ci].astype(np.float64), gy[..., :co].astype(np.float64))
    close(dW.cpu().numpy(), rW, 1e-4)
    close(db.cpu().numpy(), rb, 1e-4)


def test_restriction():
    f = np.random.default_rng(9).normal(size=(16, 24, 32)).astype(np.float32)
    c = ls.restrict4(torch.from_numpy(f).cuda()).cpu().numpy()
    assert np.max(np.abs(c - oracle.restrict4(f.astype(np.float64)))) <= 1e-6


@SHAPES
def test_conv_matches_oracle_network_forward(shape):
    """The four layers chained on the GPU against the oracle's network."""
    x = rand_act(10, 3, shape)
    r = np.random.default_rng(11)
    chans = [3, 16, 16, 16, 1]
    params = [(bf16_round(r.normal(size=(27, chans[k], chans[k + 1])) * 0.15),
               (r.normal(size=chans[k + 1]) * 0.05).astype(np.float32)) for k in range(4)]
    a = to_dev_bf16(x)
    for k, (W, b) in enumerate(params):
        a, st = ls.conv3_bf16(a, torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), 1 if k == 3 else 0)
    torch.cuda.synchronize()
    ref = oracle.cnn_forward(x[..., :3].astype(np.float64), [(W.astype(np.float64), b) for W, b in params])[-1]
    close(a.cpu().numpy(), ref[..., 0], 5e-2)
