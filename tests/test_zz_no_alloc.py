"""The velocity entry point that allocates no device memory (for callers that cannot
allocate while they need the field, e.g. during CUDA-graph capture or under a fixed
memory budget) against the context-based entry point, through the C-ABI."""
import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

pytestmark = pytest.mark.gpu

FIELD_TOL = 2e-5  # the FP32 field tolerance of the other GPU tests, relative to the field's scale


@pytest.mark.parametrize("shape", [(64, 64), (32, 128)])
def test_noalloc_velocity_matches_context_entry_point(shape):
    import torch
    Ly, Lx = shape
    m = synth.strip_map(Lx, Ly, [0, Lx // 4, Lx // 2, Lx], [1.0, 3.0, 0.5], spacing=0.6) \
        if Lx != Ly else synth.make_workload("voronoi16_64", L=Lx, n=16)
    ts = (0.0, 0.7, 25.0)
    refs = []
    with P.Cartogram(Lx, Ly, 1.0, precision="mixed") as c:
        c.set_map(m)
        spec = c.spectrum()
        for t in ts:
            refs.append(c.velocity(t)[1])
    spec = spec.copy()
    spec[0, 0] = 0.0
    dspec = torch.tensor(spec, dtype=torch.float32, device="cuda")
    out = torch.empty((Ly, Lx, 2), dtype=torch.float32, device="cuda")
    # two calls in a row per time: the shared scratch keeps the previous call's contents
    for t, ref in zip(ts, refs):
        for _ in range(2):
            out.fill_(float("nan"))
            P.cartogram_velocity_noalloc(Lx, Ly, dspec, t, out)
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            scale = max(float(np.max(np.abs(ref))), 1e-30)
            assert np.max(np.abs(got - ref)) <= FIELD_TOL * scale


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch
    spec = torch.zeros((1024, 1024), dtype=torch.float32, device="cuda")
    out = torch.empty((1024, 1024, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(P.CartogramError) as e:
        P.cartogram_velocity_noalloc(1024, 1024, spec, 1.0, out)
    assert e.value.code == P.CG_EINVAL
    with pytest.raises(P.CartogramError) as e:
        P.cartogram_velocity_noalloc(48, 64, spec, 1.0, out)
    assert e.value.code == P.CG_EINVAL
