"""eig_gram_noalloc: the Gram product for callers that cannot allocate device memory (its scratch
is a fixed array inside the library).  Its result must equal eig_gram's on the same inputs, on
two calls in a row (the shared scratch keeps the previous call's contents), and the capped
grouping of a GPU with more SMs than the array has partials must still give A^T B (against the
oracle's FP64 product).  This file is collected last so that a run stopping at the first failure
has already run every other test."""
import numpy as np
import pytest

import oracle as O

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


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
@pytest.mark.parametrize("parts", [1, 7, 300])
def test_gram_noalloc_capped_partials_match_oracle(dt, parts):
    """More rows per CTA partial than eig_gram uses here (the 512-partial cap of a larger GPU,
    forced through eig_gram_noalloc_parts), checked element by element against O.gram."""
    from paper_2305_15552_gb300 import binding
    binding.load()
    rng = np.random.default_rng(5 + parts)
    n, nb = 100003, 16
    A = torch.tensor(rng.standard_normal((n, nb)), dtype=dt, device="cuda")
    B = torch.tensor(rng.standard_normal((n, nb)), dtype=dt, device="cuda")
    got = binding.gram_noalloc(A, B, max_parts=parts).cpu().numpy()
    Ae, Be = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = O.gram(Ae, Be)
    bound = np.abs(Ae).T @ np.abs(Be)
    tol = (2.0 ** -24 * 40 if dt == torch.float32 else 2.0 ** -53 * (n + 10)) * bound + 1e-300
    assert np.all(np.abs(got - ref) <= tol)


def test_gram_noalloc_parts_rejects_bad_cap():
    from paper_2305_15552_gb300 import binding
    binding.load()
    A = torch.ones(1000, 8, device="cuda")
    for bad in (0, 513):
        with pytest.raises(binding.EigError) as e:
            binding.gram_noalloc(A, A, max_parts=bad)
        assert e.value.status == binding.EIG_EINVAL
