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

TOL64 = 1e-12  # the FP64 parity bar of the other operator tests
TOL32 = 1e-6


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


@pytest.mark.parametrize("dtype,tol", [(torch.float64, TOL64), (torch.float32, TOL32)])
def test_static_scratch_matches_apply_B_on_two_calls(tn, dtype, tol):
    m = tn.tn_mesh_create(4, 17, 0.55, 1.0)
    try:
        eta = torch.tensor(inputs.lognormal_viscosity(tn.tn_mesh_info(m, 0)["n_wedges"], 9), device="cuda")
        tn.tn_set_viscosity(m, eta)
        pinfo = tn.tn_mesh_info(m, 1)
        for call, seed in enumerate((11, 23)):  # two calls in a row with different inputs
            u = _field(tn, m, 0, seed, dtype)
            want = torch.zeros(pinfo["n_layout"], device="cuda", dtype=dtype)
            got = torch.full_like(want, float("nan"))
            tn.tn_apply_B(m, 0, u, want)
            tn.tn_apply_B_static(m, 0, u, got)
            torch.cuda.synchronize()
            w, g = want.double().cpu().numpy(), got.double().cpu().numpy()
            valid = tn.tn_mesh_canonical_index(m, 1) >= 0
            err = np.abs(g[valid] - w[valid]).max() / np.abs(w[valid]).max()
            assert err <= tol, (call, err)
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
