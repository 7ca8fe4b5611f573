"""cosmica_propagate_noalloc: propagation for callers that cannot allocate
device memory (a foreign memory pool holds the free memory, cudaFree's
implicit device synchronisation is not allowed, or every allocation must go
through an approved allocator).  Its scratch is a fixed static device array,
so it must give exactly what cosmica_propagate gives for the same inputs, on
consecutive calls that reuse the array, up to its largest accepted size.

This file is collected last so that a failure here leaves every other test
already run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _reference(params, sp, T, n, seed):
    import torch
    m = cz.Model(params)
    out = cz.ExitBuffers(sum(n))
    cz.cosmica_propagate(m.h, sp, T, n, seed, out)
    torch.cuda.synchronize()
    res = out.numpy()
    m.close()
    return res


def _noalloc(params, sp, T, n, seed):
    import torch
    out = cz.ExitBuffers(sum(n))
    cz.cosmica_propagate_noalloc(params, sp, T, n, seed, out)
    torch.cuda.synchronize()
    return out.numpy()


@pytest.mark.parametrize("precision", [cz.PREC_MIXED, cz.PREC_FP64])
def test_noalloc_matches_propagate_on_consecutive_calls(precision):
    import torch
    assert torch.cuda.is_available()
    calls = [
        (W.params(max_steps=2_000_000), W.PROTON, [0.3, 3.0, 30.0], [37, 0, 90], 17),
        (W.config3_param_sets()[4] | {"max_steps": 2_000_000.0}, W.HELIUM4, [0.5, 5.0], [64, 33], 18),
        # the largest accepted call: 1024 energies, which reach the scratch in many parameter chunks
        (W.params(max_steps=2_000_000), W.ELECTRON, W.logspace(20.0, 100.0, 1024),
         [(k % 3) for k in range(1024)], 19),
    ]
    for p, sp, T, n, seed in calls:          # two calls in a row share the static scratch
        params = cz.make_params(p, precision)
        s = cz.make_species(sp)
        got = _noalloc(params, s, T, n, seed)
        ref = _reference(params, s, T, n, seed)
        for k in ("r", "th", "ph", "lnP", "s", "steps", "status", "item"):
            assert np.array_equal(got[k], ref[k]), (precision, k)
        assert np.all(got["status"] == cz.PATH_EXIT)


def test_noalloc_rejects_sizes_beyond_its_limit():
    params = cz.make_params(W.params(), cz.PREC_MIXED)
    n_e = 1025   # COSMICA_NOALLOC_MAX_ENERGIES + 1
    out = cz.ExitBuffers(n_e)
    with pytest.raises(cz.CosmicaError) as e:
        cz.cosmica_propagate_noalloc(params, cz.make_species(W.PROTON), [1.0] * n_e, [1] * n_e, 1, out)
    assert e.value.status == cz.ERR_INVALID and "limit" in str(e.value)
