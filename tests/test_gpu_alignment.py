"""Fields that start off a 16-byte boundary.

The 3D face kernels copy each cell's coefficients with bulk asynchronous
copies when both fields are 16-byte aligned, and fall back to plain loads
otherwise; the two routes must give the same bits.  A view that starts one
element (4 or 8 bytes) into a buffer is not 16-byte aligned.  The TF32
element kernel needs aligned fields and reports misaligned ones as an error.
"""
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _offset_copy(x):
    """The same values in a view that starts one element into its buffer."""
    buf = torch.empty(x.numel() + 1, dtype=x.dtype, device=x.device)
    v = buf[1:]
    v.copy_(x)
    assert v.data_ptr() % 16 != 0
    return v


@pytest.mark.parametrize("k,cells,dtype", [(2, (6, 4, 3), torch.float64), (3, (5, 3, 3), torch.float64),
                                           (3, (5, 3, 3), torch.float32), (2, (6, 4, 3), torch.float32)])
def test_unaligned_fields_same_bits(G, k, cells, dtype):
    ext, per = (1.0, 0.2, 0.2), (1, 0, 1)
    om = O.Mesh(3, cells, ext, per, k)
    gm = G.cdg2_mesh_create(3, cells, ext, per, k)
    p = I.default_params()
    fl = G.CDG2_MINV | (G.CDG2_FP32 if dtype == torch.float32 else 0)
    U = gaussian_state(om, sigma=0.08, seed=3).reshape(-1).to("cuda", dtype)
    dU = (random_state(om, seed=4) - 1.0).reshape(-1).to("cuda", dtype)
    Uo, dUo = _offset_copy(U), _offset_copy(dU)
    for op in ("apply", "jvp"):
        a, b = torch.empty_like(U), torch.empty_like(U)
        if op == "apply":
            G.cdg2_apply(gm, p, U, a, fl)
            G.cdg2_apply(gm, p, Uo, b, fl)
        else:
            G.cdg2_jvp(gm, p, U, dU, a, fl)
            G.cdg2_jvp(gm, p, Uo, dUo, b, fl)
        assert torch.equal(a, b), (op, float((a - b).abs().max()))


def test_tf32_rejects_misaligned_fields(G):
    cells, ext, per = (5, 3, 3), (1.0, 0.2, 0.2), (1, 0, 1)
    om = O.Mesh(3, cells, ext, per, 3)
    gm = G.cdg2_mesh_create(3, cells, ext, per, 3)
    U = gaussian_state(om, sigma=0.08, seed=3).reshape(-1).to("cuda", torch.float32)
    out = torch.empty_like(U)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_apply(gm, I.default_params(), _offset_copy(U), out, G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32)
    # the mesh stays usable
    G.cdg2_apply(gm, I.default_params(), U, out, G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32)
    assert bool(torch.isfinite(out).all())
