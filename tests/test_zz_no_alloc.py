"""The allocation-free box solve matches the context-based one (kept last in collection).

kfbi_grid_solve_noalloc serves callers that cannot allocate device memory on the solve path
(a host application whose memory pool owns the device, or a loop that must not call
cudaMalloc); its scratch is a static device array shared by all calls. Two calls in a row
must each reproduce kfbi_grid_solve, so the second call must not depend on what the first
left in the shared array.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_01068_gb300.kfbi")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_01068_gb300 import build

    build.build()
    K.load()


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("N,boxbc,kappa", [(64, K.BOX_DIRICHLET0, 0.0), (512, K.BOX_NEUMANN0, 12.5),
                                           (256, K.BOX_DIRICHLET0, 40.0)])
def test_noalloc_matches_context_solve_twice(N, boxbc, kappa):
    box = (-1.0, 1.0, -1.0, 1.0)
    ctx = K.Context(N, box, kappa, boxbc, K.FP64, max_nodes=64)
    h = (box[1] - box[0]) / N
    rng = np.random.default_rng(N)
    for call in range(2):
        rhs = torch.tensor(rng.standard_normal((N, N)), dtype=torch.float64, device="cuda")
        ref = ctx.grid_solve(rhs)
        u = K.grid_solve_noalloc(rhs, h, kappa, boxbc)
        torch.cuda.synchronize()
        assert rel(u, ref) < 1e-12, f"call {call}"
    ctx.close()


def test_noalloc_rejects_sizes_beyond_maximum():
    rhs = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KfbiError) as e:
        K.grid_solve_noalloc(rhs, 1.0 / 512)
    assert e.value.status == K.ERR_CAPACITY
    with pytest.raises(K.KfbiError) as e:
        K.grid_solve_noalloc(torch.zeros((64, 64), dtype=torch.float64, device="cuda"), 0.1, 0.0, K.BOX_NEUMANN0)
    assert e.value.status == K.ERR_SINGULAR


def test_noalloc_in_place_and_on_a_side_stream():
    """rhs and u may alias; a call on a non-default stream, synchronised, gives the same result."""
    N, box, kappa = 128, (-1.0, 1.0, -1.0, 1.0), 3.0
    h = (box[1] - box[0]) / N
    ctx = K.Context(N, box, kappa, K.BOX_DIRICHLET0, K.FP64, max_nodes=64)
    rng = np.random.default_rng(7)
    rhs = torch.tensor(rng.standard_normal((N, N)), dtype=torch.float64, device="cuda")
    ref = ctx.grid_solve(rhs.clone())
    buf = rhs.clone()
    u = K.grid_solve_noalloc(buf, h, kappa, K.BOX_DIRICHLET0, out=buf)
    torch.cuda.synchronize()
    assert u.data_ptr() == buf.data_ptr()
    assert rel(u, ref) < 1e-12
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        u2 = K.grid_solve_noalloc(rhs, h, kappa, K.BOX_DIRICHLET0)
    side.synchronize()
    assert rel(u2, ref) < 1e-12
    ctx.close()


def test_noalloc_rejects_a_wrong_output_before_the_call():
    rhs = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    for bad in (torch.zeros((64, 64), dtype=torch.float32, device="cuda"),
                torch.zeros((32, 64), dtype=torch.float64, device="cuda"),
                torch.zeros((64 * 64,), dtype=torch.float64, device="cuda")):
        with pytest.raises(ValueError):
            K.grid_solve_noalloc(rhs, 1.0 / 32, out=bad)
