"""The Python binding refuses host (CPU) tensors before any library or CUDA
call: the kernels read their arguments on the GPU, where a host address
would fault."""
import pytest

torch = pytest.importorskip("torch")

import paper_2501_11592_gb300 as cs


def cpu(*shape, dtype=None):
    return torch.zeros(*shape, dtype=dtype or torch.float32)


@pytest.mark.parametrize("call", [
    lambda: cs.omp_solve_batched(cpu(4, 8), cpu(4, 2), 2),
    lambda: cs.clomp_solve_batched(cpu(4, 8), cpu(4, 2), 2),
    lambda: cs.iht_solve_batched(cpu(4, 8), cpu(4, 2), 2, 0.5),
    lambda: cs.omp_solve(cpu(4, 8), cpu(4), 2),
    lambda: cs.correlate(cpu(4, 8), cpu(4, 2)),
    lambda: cs.synthesize(None, cpu(2, 3, dtype=torch.int32), cpu(2, 3), cpu(2, dtype=torch.int32), n=8),
    lambda: cs.image_quality(cpu(16, 32), cpu(16, 32), 16),
    lambda: cs.clfit_forward(cpu(4, 8), cpu(2, 3, dtype=torch.int32), cpu(2, 3), cpu(4, 2)),
    lambda: cs.clfit_adjoint(cpu(4, 8), cpu(2, 3, dtype=torch.int32), cpu(4, 2)),
    lambda: cs.omp_solve_varlen([(cpu(4, 8), cpu(4), 2)]),
    lambda: cs.clomp_solve_varlen([(cpu(4, 8), cpu(4), 2)]),
])
def test_host_tensors_are_refused(call):
    with pytest.raises(ValueError, match="CUDA tensors"):
        call()
