"""The velocity entry point that allocates no device memory, through the C-ABI.

Some callers of this library cannot allocate GPU memory when they need the field: a
host application that gives the library a fixed device-memory budget and owns every
allocation itself, or a real-time loop that must not call the allocator. For them
cartogram_velocity_noalloc keeps its scratch in a fixed device array. These tests
check it against the context-based entry point and against the FP64 oracle, on two
calls in a row (the shared scratch keeps the previous call's contents), and check
that it rejects sizes beyond its maximum and misaligned or foreign pointers before
any kernel runs. The file is collected last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import paper_1802_07625_gb300 as P
from paper_1802_07625_gb300 import synth

pytestmark = pytest.mark.gpu

FIELD_TOL = 2e-5  # the FP32 field tolerance of the other GPU tests, relative to the field's scale


def _map(Lx, Ly):
    if Lx != Ly:
        return synth.strip_map(Lx, Ly, [0, Lx // 4, Lx // 2, Lx], [1.0, 3.0, 0.5], spacing=0.6)
    return synth.make_workload("voronoi16_64", L=Lx, n=16)


@pytest.mark.parametrize("shape", [(64, 64), (32, 128)])
def test_noalloc_velocity_matches_context_entry_point(shape):
    import torch
    Ly, Lx = shape
    m = _map(Lx, Ly)
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


def test_noalloc_velocity_matches_oracle(orc):
    """The field of the FP32 spectrum the call receives, against the oracle's direct
    cosine/sine sums (SI Eq. rhoxyt) and Fick's law v = -grad(rho)/rho in FP64."""
    import torch
    Lx = Ly = 64
    m = _map(Lx, Ly)
    with P.Cartogram(Lx, Ly, 1.0, precision="mixed") as c:
        c.set_map(m)
        spec = c.spectrum()
    spec = spec.copy()
    spec[0, 0] = 0.0
    spec32 = spec.astype(np.float32)
    dspec = torch.tensor(spec32, device="cuda")
    # the oracle evaluates the same (FP32-rounded) coefficients, with the mean restored
    ospec = spec32.astype(np.float64)
    ospec[0, 0] = Lx * Ly
    out = torch.empty((Ly, Lx, 2), dtype=torch.float32, device="cuda")
    for t in (0.0, 0.7, 25.0):
        vx, vy, _ = orc.velocity(*orc.fields(ospec, t))
        scale = max(float(np.max(np.hypot(vx, vy))), 1e-30)
        for _ in range(2):
            out.fill_(float("nan"))
            P.cartogram_velocity_noalloc(Lx, Ly, dspec, t, out)
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            assert np.max(np.abs(got[..., 0] - vx)) <= 4 * FIELD_TOL * scale
            assert np.max(np.abs(got[..., 1] - vy)) <= 4 * FIELD_TOL * scale


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


def test_noalloc_rejects_misaligned_and_host_pointers():
    """The field is written with 16-byte stores: an output 8 bytes off a 16-byte boundary
    is refused before any launch, as are host buffers."""
    import torch
    Lx = Ly = 64
    spec = torch.zeros((Ly, Lx), dtype=torch.float32, device="cuda")
    buf = torch.zeros(2 * Lx * Ly + 4, dtype=torch.float32, device="cuda")
    shifted = buf[2:2 + 2 * Lx * Ly]  # contiguous, 8 bytes past an aligned base
    assert shifted.data_ptr() % 16 == 8
    with pytest.raises(P.CartogramError) as e:
        P.cartogram_velocity_noalloc(Lx, Ly, spec, 1.0, shifted)
    assert e.value.code == P.CG_EINVAL
    assert torch.all(buf == 0)
    host = np.zeros((Ly, Lx, 2), dtype=np.float32)
    rc = P.load().cartogram_velocity_noalloc(Lx, Ly, spec.data_ptr(), 1.0, host.ctypes.data, None)
    assert rc == P.CG_EINVAL
    with pytest.raises(ValueError):
        P.cartogram_velocity_noalloc(Lx, Ly, spec, 1.0, buf[:16])
