"""fftc_execute allocates and synchronises nothing, so a call can be captured into a CUDA
graph on the caller's stream and replayed (the replay reuses the buffers given at capture):
one-pass, four-step, tensor-core, mixed-radix, FP64 and multidimensional plans, each replay
bit-identical to a direct execute and within tolerance of the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synthetic_inputs as si
from gpu_util import from_device, rel_l2_rows, to_device, tol_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2308_00497_gb300 import build
    build.build()


def _dev(x, layout, fp64):
    if fp64:
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128))).cuda()
    return to_device(x, layout)


def _host(t, layout, fp64):
    return t.cpu().numpy() if fp64 else from_device(t, layout)


def _captured(run, x):
    """A graph holding run(x, out) (after one warm-up call outside the capture) and out."""
    out = torch.empty_like(x)
    run(x, out)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run(x, out)
    return g, out


@pytest.mark.parametrize("n,layout,precision,tol", [
    (1024, "interleaved", "fp32", None), (1 << 14, "split", "fp32", None), (1 << 17, "interleaved", "fp32", None),
    (1 << 20, "split", "fp32", None), (1 << 13, "interleaved", "fp16_tc_split", 1e-4),
    (1000, "interleaved", "fp32", None), (6000, "split", "fp32", None), (1024, "interleaved", "fp64", 1e-13)])
def test_execute_replays_from_a_cuda_graph(n, layout, precision, tol):
    import paper_2308_00497_gb300 as fc
    B = max(2, min(64, (1 << 21) // n))
    fp64 = precision == "fp64"
    p = fc.Plan(n, B, layout, False, precision)
    x0 = si.uniform_complex(B, n, seed=n % 97)
    x1 = si.uniform_complex(B, n, seed=n % 97 + 1)
    xd = _dev(x0, layout, fp64)
    g, out = _captured(lambda a, b: p.execute(a, b), xd)
    new = _dev(x1, layout, fp64)
    xd.copy_(new)
    g.replay()
    direct = p.execute(new)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(out) if out.is_complex() else out,
                       torch.view_as_real(direct) if direct.is_complex() else direct)
    ref = oracle.fft(x1.astype(np.complex128))
    assert rel_l2_rows(_host(out, layout, fp64), ref).max() <= (tol if tol else tol_fp32(n))


def test_nd_execute_replays_from_a_cuda_graph():
    import paper_2308_00497_gb300 as fc
    dims, B = (64, 128), 3
    x0 = si.uniform_complex(B, dims[0] * dims[1], seed=7).reshape(B, *dims)
    x1 = si.uniform_complex(B, dims[0] * dims[1], seed=8).reshape(B, *dims)
    p = fc.NdPlan(dims, B, "interleaved", False)
    xd = torch.from_numpy(np.ascontiguousarray(x0.astype(np.complex64))).cuda()
    g, out = _captured(lambda a, b: p.execute(a, b), xd)
    xd.copy_(torch.from_numpy(np.ascontiguousarray(x1.astype(np.complex64))).cuda())
    g.replay()
    torch.cuda.synchronize()
    ref = oracle.fftn(x1.astype(np.complex128), rank=2)
    err = rel_l2_rows(out.cpu().numpy().reshape(B, -1), ref.reshape(B, -1)).max()
    assert err <= tol_fp32(dims[0] * dims[1])
