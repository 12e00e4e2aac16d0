"""The projection entry point for callers that cannot allocate device memory.

Some users embed this library where allocating GPU memory is forbidden after
start-up (a host program that owns every device buffer, or a loop with hard
latency limits).  sdf_project_noalloc serves them from a scratch array built
into the library.  This file is collected last on purpose, so that a run that
stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2606_17971_b300 import sdf  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("n,k", [((83, 41), 37), ((200, 130), 128)])
def test_noalloc_projection_matches_workspace_projection_on_two_calls(n, k):
    rng = np.random.default_rng(2024 + k)
    N = n[0] * n[1]
    G = sdf.Problem(2, n)
    Phi = rng.standard_normal((k, N))
    G.set_modes(torch.as_tensor(Phi, dtype=torch.float64, device=DEV))
    out = torch.empty(k, dtype=torch.float64, device=DEV)
    for call in range(2):  # the second call sees the first call's leftovers
        act = rng.random(N) < (0.2 + 0.3 * call)
        v = rng.standard_normal(N) * (1 + 10 * call)
        act_t = torch.as_tensor(act.astype(np.uint8), device=DEV)
        v_t = torch.as_tensor(v, dtype=torch.float64, device=DEV)
        ref = G.project(act_t, v_t).cpu().numpy()
        got = G.project_noalloc(act_t, v_t, out).cpu().numpy()
        scale = np.abs(Phi).sum(1).max() * np.abs(v).max()
        assert np.max(np.abs(got - ref)) <= 1e-12 * scale
        assert np.max(np.abs(got - Phi[:, ~act] @ v[~act])) <= 1e-12 * scale
