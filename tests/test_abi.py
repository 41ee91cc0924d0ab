"""Host-side checks that need no GPU: the C-ABI library builds, loads and exports every
entry point that include/cartogram.h declares, and the Python binding covers them."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cartogram.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cartogram_\w+)\s*\(", src)))


def test_header_declares_the_method_calls():
    names = _declared()
    for n in ("cartogram_init", "cartogram_set_regions", "cartogram_integrate", "cartogram_project",
              "cartogram_area_errors", "cartogram_destroy", "cartogram_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import ctypes

    import paper_1802_07625_gb300 as P
    P.load()
    lib = ctypes.CDLL(P.library_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_a_function_per_entry_point():
    import paper_1802_07625_gb300 as P
    for n in _declared():
        assert callable(getattr(P, n)), n


def test_default_options_without_gpu():
    import paper_1802_07625_gb300 as P
    o = P.cartogram_default_options()
    assert o.precision == P.CG_PRECISION_FP64
    assert o.dt0 == 1e-2 and o.atol == 1e-2 and o.grow == 1.2 and o.shrink == 0.5
    assert o.cfl == 1.0 and o.rho_tol == 1e-4 and o.area_tol == 0.01
    assert o.max_steps == 4000 and o.max_iter == 500 and o.use_graph == 1 and o.blur_decay == 0.5 and o.autotune == 1
    assert o.flow == P.CG_FLOW_DIFFUSION and o.time_limit == 0.0
    assert o.barrier_spins == 1 << 25


def test_binding_structs_match_the_header_layout(tmp_path):
    # compile a probe against the header and compare every field offset and the sizes
    import ctypes
    import shutil
    import subprocess

    import paper_1802_07625_gb300 as P
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = []
    for struct, cls in (("cg_options", P.Options), ("cg_stats", P.Stats)):
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (struct, struct))
        for name, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (struct, name, struct, name))
    src = tmp_path / "probe.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "cartogram.h"\nint main(void) {\n' +
                   "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for struct, cls in (("cg_options", P.Options), ("cg_stats", P.Stats)):
        assert got[(struct, "sizeof")] == ctypes.sizeof(cls), struct
        for name, _ in cls._fields_:
            assert got[(struct, name)] == getattr(cls, name).offset, (struct, name)


def test_init_rejects_bad_sizes_before_touching_the_gpu():
    import paper_1802_07625_gb300 as P
    for Lx, Ly in ((0, 64), (64, 48), (2048, 64), (4, 4)):
        with pytest.raises(P.CartogramError) as e:
            P.cartogram_init(Lx, Ly, 1.0)
        assert e.value.code == P.CG_EINVAL
    with pytest.raises(P.CartogramError) as e:
        P.cartogram_init(64, 64, -1.0)
    assert e.value.code == P.CG_EINVAL
    o = P.cartogram_default_options()
    o.flow = 2
    with pytest.raises(P.CartogramError) as e:
        P.cartogram_init(64, 64, 1.0, o)
    assert e.value.code == P.CG_EINVAL
    for bad in (-1.0, float("nan"), float("inf")):
        o = P.cartogram_default_options()
        o.time_limit = bad
        with pytest.raises(P.CartogramError) as e:
            P.cartogram_init(64, 64, 1.0, o)
        assert e.value.code == P.CG_EINVAL
    for bad in (0, -5, (1 << 40) + 1):
        o = P.cartogram_default_options()
        o.barrier_spins = bad
        with pytest.raises(P.CartogramError) as e:
            P.cartogram_init(64, 64, 1.0, o)
        assert e.value.code == P.CG_EINVAL


def test_oracle_and_library_share_no_source():
    # the oracle is independent of the CUDA path: no include, import or file in common
    orc = open(os.path.join(ROOT, "oracle", "cartogram_oracle.c")).read()
    assert "#include \"" not in orc
    csrc = os.path.join(ROOT, "paper_1802_07625_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower(), f
    for f in ("__init__.py", "build.py", "synth.py"):
        txt = open(os.path.join(ROOT, "paper_1802_07625_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def test_unknown_options_are_rejected_before_touching_the_gpu():
    import paper_1802_07625_gb300 as P
    with pytest.raises(TypeError):
        P.Cartogram(64, 64, 1.0, no_such_option=1)
    with pytest.raises(ValueError):
        P.Cartogram(64, 64, 1.0, flow="sideways")
    o = P.cartogram_default_options()
    for name in ("time_limit", "max_iter", "blur_decay", "use_graph", "autotune", "flow"):
        assert hasattr(o, name)
