"""GPU parity of lap5_apply against the oracle's stencil (Sec. II-B mask).

The GPU kernel and the oracle use the same fixed add order, so binary64,
binary32 and bf16 results must be bit-identical, on ragged shapes, on
unaligned pitches (scalar path), and at the full 8192 x 8192 size.
"""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 9), (9, 1), (2, 2), (3, 5), (63, 65), (64, 64), (65, 33), (127, 130), (129, 7), (1000, 37),
          (257, 300), (513, 19), (2049, 17)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("pitch", ["tight", "aligned", "wide"])
def test_f64_bit_exact(nx, ny, pitch):
    ld = {"tight": nx, "aligned": gen.pitch(nx, 8), "wide": gen.pitch(nx, 8) + 6}[pitch]
    x = gen.uniform_rhs(nx, ny, seed=nx * 7 + ny, ld=ld)
    x[:, nx:] = 99.0
    y = lap5cg.lap5_apply(_dev(x), nx=nx).cpu().numpy()
    ref = oracle.lap5_apply(x, nx=nx)
    np.testing.assert_array_equal(y[:, :nx], ref[:, :nx])
    assert not y[:, nx:].any()  # padding untouched (the output started at zero)


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("pitch", ["tight", "aligned"])
def test_f32_bit_exact(nx, ny, pitch):
    ld = nx if pitch == "tight" else gen.pitch(nx, 4)
    x = gen.uniform_rhs(nx, ny, seed=nx + 3 * ny, ld=ld, dtype=np.float32)
    y = lap5cg.lap5_apply(_dev(x), nx=nx).cpu().numpy()
    ref = oracle.lap5_apply(x, nx=nx, dtype=np.float32)
    np.testing.assert_array_equal(y[:, :nx], ref[:, :nx])


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (7, 16), (8, 300), (64, 64), (129, 70), (256, 16), (256, 33),
                                   (264, 1), (300, 257), (513, 19), (1000, 37), (2049, 17)])
@pytest.mark.parametrize("pitch", ["tight", "aligned", "quad", "wide"])
def test_bf16_bit_exact(nx, ny, pitch):
    # aligned / wide: ld a multiple of 8 (TMA tiles of 16 rows x 256 columns,
    # the zero fill standing for every operand outside the grid); quad:
    # ld = 4 mod 8 (four columns a lane); tight: scalar accesses
    ld = {"tight": nx, "aligned": gen.pitch(nx, 2), "quad": gen.pitch(nx, 2) + 4, "wide": gen.pitch(nx, 2) + 24}[pitch]
    xf = gen.uniform_rhs(nx, ny, seed=nx + ny, ld=ld, dtype=np.float32)
    xb = oracle.f32_to_bf16_bits(xf)
    xb[:, nx:] = 0x4049  # padding (3.14) must not leak into the result
    xt = torch.from_numpy(xb.view(np.int16)).to("cuda").view(torch.bfloat16)
    y = lap5cg.lap5_apply(xt, nx=nx).view(torch.int16).cpu().numpy().view(np.uint16)
    ref = oracle.lap5_apply(xb, nx=nx, dtype="bf16")
    np.testing.assert_array_equal(y[:, :nx], ref[:, :nx])
    assert not y[:, nx:].any()  # padding untouched (the output started at zero)


def test_eigenvector_closed_form_on_gpu():
    nx, ny = 300, 200
    v = gen.sine_mode(nx, ny, 3, 5, ld=gen.pitch(nx, 8))
    lam = gen.mode_eigenvalue(nx, ny, 3, 5)
    y = lap5cg.lap5_apply(_dev(v), nx=nx).cpu().numpy()
    assert np.abs(y[:, :nx] - lam * v[:, :nx]).max() <= 8e-14


@pytest.mark.parametrize("n", [4096, 8192])
def test_full_size_f64(n):
    x = gen.uniform_rhs(n, n, seed=3)
    y = lap5cg.lap5_apply(_dev(x)).cpu().numpy()
    ref = oracle.lap5_apply(x)
    np.testing.assert_array_equal(y, ref)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_full_size_8192_narrow_types(dtype):
    # binary32 runs eight columns a lane (two 16-byte groups), bf16 sixteen
    n = 8192
    xf = gen.uniform_rhs(n, n, seed=4, dtype=np.float32)
    if dtype == "f32":
        y = lap5cg.lap5_apply(_dev(xf)).cpu().numpy()
        ref = oracle.lap5_apply(xf, dtype=np.float32)
    else:
        xb = oracle.f32_to_bf16_bits(xf)
        xt = torch.from_numpy(xb.view(np.int16)).to("cuda").view(torch.bfloat16)
        y = lap5cg.lap5_apply(xt).view(torch.int16).cpu().numpy().view(np.uint16)
        ref = oracle.lap5_apply(xb, dtype="bf16")
    np.testing.assert_array_equal(y, ref)


def test_output_stream_ordering():
    # the call is asynchronous on the given stream
    s = torch.cuda.Stream()
    x = _dev(gen.uniform_rhs(512, 512, seed=1))
    with torch.cuda.stream(s):
        y = lap5cg.lap5_apply(x, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), oracle.lap5_apply(x.cpu().numpy()))
