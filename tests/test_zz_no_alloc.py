"""sem_dot_noalloc: the inner product for callers that cannot let the library
allocate device memory (a fixed device-memory budget, or a loop that cannot
pay for cudaMalloc/cudaFree).  Its reduction scratch is a static device array,
so two calls in a row must both agree with sem_dot, whose scratch the mesh
allocated.  Collected last so that a run stopping at the first failure has
run every other test first."""

import numpy as np
import pytest

from paper_2110_01716_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_01716_gb300 import sem  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2110_01716_gb300 import build

    build.build()


@pytest.mark.parametrize("ex,ey,ez,N", [(3, 2, 4, 3), (8, 8, 8, 7), (5, 7, 9, 7), (1, 1, 1, 1)])
def test_noalloc_dot_matches_sem_dot_on_two_calls(ex, ey, ez, N):
    m = sem.Mesh(ex, ey, ez, N, sem.SEM_DIRICHLET, verts=inputs.box_vertices(ex, ey, ez, 0.1, 2))
    u = torch.tensor(inputs.random_field(m.n_local, 1), device=DEV)
    v = torch.tensor(inputs.random_field(m.n_local, 2), device=DEV)
    ref = sem.sem_dot(m, u, v)
    scale = np.sqrt(sem.sem_dot(m, u, u) * sem.sem_dot(m, v, v))
    out = torch.full((1,), float("nan"), device=DEV, dtype=torch.float64)
    for _ in range(2):
        out.fill_(float("nan"))
        sem.sem_dot_noalloc(m, u, v, out)
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= 1e-12 * scale, (out.item(), ref)
    # a different pair right after: the shared scratch carries nothing over
    w = torch.tensor(inputs.random_field(m.n_local, 3), device=DEV)
    sem.sem_dot_noalloc(m, w, v, out)
    torch.cuda.synchronize()
    ref2 = sem.sem_dot(m, w, v)
    assert abs(out.item() - ref2) <= 1e-12 * np.sqrt(sem.sem_dot(m, w, w) * sem.sem_dot(m, v, v))


def test_noalloc_dot_rejects_meshes_beyond_its_scratch():
    # 64 x 64 x 33 elements at N = 7: 69.2 M local points > 67,092,480
    m = sem.Mesh(64, 64, 33, 7, sem.SEM_DIRICHLET, sem.SEM_GEOM_TRILINEAR, jitter=0.0)
    u = torch.zeros(1, device=DEV, dtype=torch.float64)
    out = torch.zeros(1, device=DEV, dtype=torch.float64)
    # the library's own check, through the C ABI (the binding would reject
    # these short tensors before the call)
    with pytest.raises(sem.SemError) as ei:
        sem.check(sem.lib().sem_dot_noalloc(m.h, sem._ptr(u), sem._ptr(u), sem._ptr(out), None))
    assert ei.value.status == sem.SEM_EINVAL
    assert "at most" in str(ei.value)
    # the binding checks the tensors it is given
    with pytest.raises(ValueError):
        sem.sem_dot_noalloc(m, u, u, out)
    small = sem.Mesh(2, 2, 2, 3, sem.SEM_DIRICHLET, verts=inputs.box_vertices(2, 2, 2, 0.1, 2))
    v = torch.zeros(small.n_local, device=DEV, dtype=torch.float64)
    with pytest.raises(ValueError):
        sem.sem_dot_noalloc(small, v, v, torch.zeros(1, device=DEV, dtype=torch.float32))
