"""eig_gram_noalloc: the Gram product for callers that cannot allocate device memory (its scratch
is a fixed array inside the library).  Its result must equal eig_gram's on the same inputs, on
two calls in a row (the shared scratch keeps the previous call's contents).  This file is
collected last so that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_gram_noalloc_matches_gram_on_two_calls(dt):
    from paper_2305_15552_gb300 import binding
    binding.load()
    rng = np.random.default_rng(11)
    for call, (n, nb) in enumerate([(200003, 16), (70001, 8)]):
        A = torch.tensor(rng.standard_normal((n, nb)), dtype=dt, device="cuda")
        B = torch.tensor(rng.standard_normal((n, nb)), dtype=dt, device="cuda")
        ref = binding.gram(A, B).cpu().numpy()
        got = binding.gram_noalloc(A, B).cpu().numpy()
        torch.cuda.synchronize()
        Ae, Be = A.double().cpu().numpy(), B.double().cpu().numpy()
        bound = np.abs(Ae).T @ np.abs(Be)
        tol = (2.0 ** -24 * 40 if dt == torch.float32 else 2.0 ** -53 * (n + 10)) * bound + 1e-300
        assert np.all(np.abs(got - ref) <= tol), f"call {call}"


def test_gram_noalloc_rejects_oversized_block():
    from paper_2305_15552_gb300 import binding
    binding.load()
    A = torch.ones(1000, 64, device="cuda")
    with pytest.raises(binding.EigError) as e:
        binding.gram_noalloc(A, A)
    assert e.value.status == binding.EIG_EINVAL
