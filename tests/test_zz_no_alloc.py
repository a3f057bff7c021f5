"""tn_apply_B_static against tn_apply_B, through the C ABI.

tn_apply_B_static is for callers that cannot allocate device memory where they call it (for
instance under an allocator that forbids cudaMalloc after start-up): its fine-level scratch is a
static device array in the library instead of mesh-owned memory.  It must give the same
divergence as tn_apply_B, on consecutive calls that reuse the shared array, and refuse levels
whose scratch does not fit in the array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2609_21633_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_21633_gb300 as tn
    tn.lib()
    return tn


def _field(tn, m, level, seed, dtype):
    info = tn.tn_mesh_info(m, level)
    canon = tn.tn_mesh_canonical_index(m, level)
    out = []
    for c in range(3):
        v = inputs.normal(info["n_layout"], seed + c)
        v = np.where(canon >= 0, v[np.maximum(canon, 0)], 0.0)
        out.append(torch.tensor(v, device="cuda", dtype=dtype))
    return out


def _mesh_with_viscosity(tn, level, n_r, seed):
    m = tn.tn_mesh_create(level, n_r, 0.55, 1.0)
    eta = torch.tensor(inputs.lognormal_viscosity(tn.tn_mesh_info(m, 0)["n_wedges"], seed), device="cuda")
    tn.tn_set_viscosity(m, eta)
    return m


def _fill_static_array_with_other_data(tn, dtype):
    """A call on a different mesh shape leaves unrelated, non-zero data in the shared array."""
    other = _mesh_with_viscosity(tn, 3, 33, 5)
    try:
        q = torch.zeros(tn.tn_mesh_info(other, 1)["n_layout"], device="cuda", dtype=dtype)
        tn.tn_apply_B_static(other, 0, _field(tn, other, 0, 77, dtype), q)
        torch.cuda.synchronize()
    finally:
        tn.tn_mesh_destroy(other)


# level 4 runs the haloed tile kernels; level 5 in FP64 the halo-free tiles with the mesh's ring buffer
@pytest.mark.parametrize("level,n_r", [(4, 17), (5, 9)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_static_scratch_matches_apply_B_bitwise_on_two_calls(tn, level, n_r, dtype):
    """Same kernels, same reduction order: the result must equal tn_apply_B's bit for bit on every
    real layout entry, on two calls in a row with different inputs, after the array was left
    holding another shape's data."""
    _fill_static_array_with_other_data(tn, dtype)
    m = _mesh_with_viscosity(tn, level, n_r, 9)
    try:
        pinfo = tn.tn_mesh_info(m, 1)
        valid = torch.tensor(tn.tn_mesh_canonical_index(m, 1) >= 0, device="cuda")
        for call, seed in enumerate((11, 23)):
            u = _field(tn, m, 0, seed, dtype)
            want = torch.zeros(pinfo["n_layout"], device="cuda", dtype=dtype)
            got = torch.full_like(want, float("nan"))
            tn.tn_apply_B(m, 0, u, want)
            tn.tn_apply_B_static(m, 0, u, got)
            torch.cuda.synchronize()
            assert torch.equal(got[valid], want[valid]), (call, (got[valid] - want[valid]).abs().max().item())
            assert want[valid].abs().max().item() > 0
    finally:
        tn.tn_mesh_destroy(m)


def test_static_scratch_rejects_levels_beyond_its_size(tn):
    m = tn.tn_mesh_create(7, 9, 0.55, 1.0, max_levels=2)  # 10 x 9 x 129 x 132 doubles > 8 MiB
    try:
        tn.tn_set_viscosity(m, torch.ones(tn.tn_mesh_info(m, 0)["n_wedges"], device="cuda", dtype=torch.float64))
        u = [torch.zeros(tn.tn_mesh_info(m, 0)["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
        q = torch.zeros(tn.tn_mesh_info(m, 1)["n_layout"], device="cuda", dtype=torch.float64)
        with pytest.raises(tn.TnError) as e:
            tn.tn_apply_B_static(m, 0, u, q)
        assert e.value.status == tn.TN_EINVAL and "static scratch" in str(e.value)
    finally:
        tn.tn_mesh_destroy(m)
