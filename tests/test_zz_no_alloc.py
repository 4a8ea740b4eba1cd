"""The allocation-free Kramers-Kronig entry point against the regular one.

apic_kk_spectra_noalloc serves callers that cannot allocate device memory
when they call (hosts that own all device memory through their own pool, or
fixed-latency loops where a cudaMalloc could stall the device). It computes
the same spectra as apic_kk_spectra from a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from helpers import as_complex, make_tiles
from paper_2407_20469_gb300 import apic, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_20469_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def _regular(plan, I):
    out = torch.zeros((I.shape[0], plan.info.n_bf, 2 * plan.info.n_pupil), dtype=torch.float32, device="cuda")
    plan.kk_spectra(I.shape[0], I, out)
    return out


@pytest.mark.parametrize("n,count", [(128, 3), (256, 2)])
def test_noalloc_kk_spectra_match_regular_entry_point_on_two_calls(n, count):
    plan = apic.Plan.from_illumination(n, synth.illumination(), max_tiles=count)
    for call, seed in enumerate((501, 502)):          # two calls in a row, different inputs
        I = torch.from_numpy(make_tiles(n, count, seed=seed + n)[0]).cuda()
        ref = _regular(plan, I)
        out = torch.full_like(ref, float("nan"))
        torch.cuda.synchronize()
        free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        plan.kk_spectra_noalloc(count, I, out)
        torch.cuda.synchronize()
        # the call allocated nothing: neither device memory as a whole nor torch's pool moved
        assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == used0, f"call {call}"
        a, b = as_complex(out), as_complex(ref)
        assert np.all(np.isfinite(a)), f"call {call}: unwritten output"
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err < 1e-6, f"call {call}: relative difference {err:.2e}"


def test_noalloc_wrapper_refuses_short_buffers():
    plan = apic.Plan.from_illumination(64, synth.illumination(), max_tiles=1)
    I = torch.zeros((1, 24, 64, 64), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, 8, 2 * plan.info.n_pupil), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        plan.kk_spectra_noalloc(2, I, out)                 # two tiles in buffers of one


def test_noalloc_rejects_host_only_plan():
    plan = apic.Plan.from_illumination(64, synth.illumination(), flags=apic.APIC_HOST_ONLY)
    with pytest.raises(apic.ApicError) as e:
        plan.kk_spectra_noalloc(1, 0, 0, stream=0)
    assert e.value.code == apic.APIC_EINVAL
