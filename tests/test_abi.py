"""Host-only checks of the C ABI library (no GPU needed): it builds, loads,
exports every function include/*.h declares, and its host-side integer
artefacts (checkpoint action lists, padded extents) agree bit for bit with
the oracle's independent generators."""
import glob
import os
import re

import pytest

from oracle import schedule as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:llg_status|long long|size_t|int|void|const char\s*\*)\s*\**\s*(\w+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2411_19109_gb300 import load
    return load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("llg_create", "llg_forward", "llg_adjoint", "levelset_step", "llg_destroy"):
        assert n in names


def test_library_exports_every_declared_function(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_names_match_the_c_names():
    import paper_2411_19109_gb300 as pkg
    from paper_2411_19109_gb300 import llg
    for name in declared_functions() - {"llg_abi_version"}:
        assert hasattr(llg, name), f"binding lacks {name}"
    assert set(llg.EXPORTED) <= declared_functions()
    assert callable(pkg.llg_forward)


@pytest.mark.parametrize("N,seg", [(1, 0), (2, 0), (17, 0), (100, 0), (101, 3), (20000, 0), (10000, 0),
                                   (50, 50), (50, 80), (9, 1)])
def test_schedule_matches_oracle(lib, N, seg):
    from paper_2411_19109_gb300 import LLG_CKPT_PERIODIC, LLG_CKPT_STORE_ALL, llg_schedule
    assert llg_schedule(N, LLG_CKPT_PERIODIC, seg) == S.periodic(N, seg)
    assert llg_schedule(N, LLG_CKPT_STORE_ALL, 0) == S.store_all(N)


@pytest.mark.parametrize("N,snaps", [(1, 0), (2, 0), (3, 1), (10, 0), (10, 2), (17, 3), (100, 1), (1000, 10),
                                     (10000, 0), (50000, 64), (7, 30)])
def test_binomial_schedule_matches_oracle(lib, N, snaps):
    from paper_2411_19109_gb300 import LLG_CKPT_BINOMIAL, llg_schedule
    assert llg_schedule(N, LLG_CKPT_BINOMIAL, snaps) == S.binomial(N, snaps)


def test_padded_extents(lib):
    from paper_2411_19109_gb300 import llg_padded_extents
    for nx, ny in [(4, 1), (32, 32), (36, 20), (128, 64), (512, 128), (1024, 512)]:
        px, py = llg_padded_extents(nx, ny)
        # linear (non-circular) convolution needs P >= 2N - 1; powers of two
        assert px >= 2 * nx - 1 and py >= 2 * ny - 1
        assert px & (px - 1) == 0 and py & (py - 1) == 0


def test_schedule_rejects_bad_arguments(lib):
    from paper_2411_19109_gb300 import LLGError, llg_schedule
    with pytest.raises(LLGError):
        llg_schedule(-1)


def test_rbf_entry_points_reject_invalid_layouts_before_device_work(lib):
    from paper_2411_19109_gb300 import LLGError, llg_rbf_phi, llg_rbf_workspace_bytes, make_rbf
    good = make_rbf(20, 12, 5e-9, 5e-9, (2, 14, 1, 10), 4, 3)
    assert llg_rbf_workspace_bytes(good) == 8 * (4 * 12 * 9 + 2 * 12 + 7)
    for bad in (make_rbf(20, 12, 5e-9, 5e-9, (2, 21, 1, 10), 4, 3),     # box beyond the grid
                make_rbf(20, 12, 5e-9, 5e-9, (5, 5, 1, 10), 4, 3),      # empty box
                make_rbf(20, 12, 5e-9, 5e-9, (2, 14, 1, 10), 0, 3),     # no RBFs
                make_rbf(20, 12, 5e-9, 5e-9, (2, 14, 1, 10), 4, 3, 0.5)):  # p < 1
        assert llg_rbf_workspace_bytes(bad) == 0
        with pytest.raises(LLGError):
            llg_rbf_phi(bad, 1, 1, 0, 1)


def test_binding_structs_have_the_c_layout(tmp_path):
    """Size and every field offset of the ctypes structs equal the C
    compiler's for include/llg.h (the spectral fields sit after penalty_w)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2411_19109_gb300 import llg as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [("llg_problem", B.llg_problem), ("llg_options", B.llg_options), ("llg_rbf", B.llg_rbf),
               ("llg_launch", B.llg_launch)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "llg.h"', "int main(void) {"]
    expect = []
    for cname, py in structs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(py))
        for f in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f[0]}));')
            expect.append(getattr(py, f[0]).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_spectral_fields_reach_the_struct():
    from paper_2411_19109_gb300 import llg as B
    import workloads as W
    p = W.random_small(8, 4, 1, objective=W.J_SPECTRAL, freqs=(8e9, 9e9), n_from=3).problem
    s = B.to_struct(p)
    assert (s.objective, s.nfreq, s.n_from) == (2, 2, 3)
    assert list(s.freqs[:2]) == [8e9, 9e9] and list(s.freqs[2:]) == [0.0] * 6
    s9 = B.to_struct(p.replace(freqs=tuple(range(1, 10))))
    assert s9.nfreq == 9 and list(s9.freqs) == list(range(1, 9))   # the library rejects nfreq > 8


def test_bench_fft_flop_model_and_reference_arm_line():
    """bench.py's host-side pieces: the FFT flop model of the FP64 roofline
    (5 N log2 N per complex transform) and the reference arm's JSON line,
    run on this host's cores on a short sample."""
    import json
    import subprocess
    import sys
    import bench
    import workloads as W
    inst = W.random_small(8, 4, 1)                   # Px = 16 -> 8-point rows; Py = 8
    assert bench.fft_flops([inst], 1) == 8 * 6 * 5 * 8 * 3
    assert bench.fft_flops([inst], 0) == 4 * 6 * 5 * 8 * 3
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, check=True, timeout=600).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "node-steps/s"
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_cuda_dormand_prince_tableau_meets_the_order_conditions(tmp_path):
    """The tableau the CUDA path compiles (csrc/dopri.cuh), printed by a host
    program and checked against the order conditions of the 5(4) pair."""
    import shutil
    import subprocess
    import numpy as np
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "tab.cu"
    src.write_text('#include <cstdio>\n#include "dopri.cuh"\nint main() {\n'
                   '  for (int s = 1; s <= 7; ++s) std::printf("%.17g\\n", llg::dp::c(s));\n'
                   '  for (int s = 1; s <= 7; ++s) for (int j = 1; j <= 7; ++j) std::printf("%.17g\\n", llg::dp::a(s, j));\n'
                   '  for (int s = 1; s <= 7; ++s) std::printf("%.17g\\n", llg::dp::b(s));\n'
                   '  for (int s = 1; s <= 7; ++s) std::printf("%.17g\\n", llg::dp::e(s));\n  return 0;\n}\n')
    exe = tmp_path / "tab"
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "paper_2411_19109_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True, capture_output=True, timeout=300)
    v = np.array([float(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                                    text=True).stdout.split()])
    c, a, b, e = v[:7], v[7:56].reshape(7, 7), v[56:63], v[63:70]
    bs = b - e
    assert np.all(np.triu(a) == 0)                                  # explicit
    np.testing.assert_allclose(a.sum(1), c, atol=1e-15)
    np.testing.assert_array_equal(a[6], b)                          # first same as last
    for w, order in ((b, 5), (bs, 4)):
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        for q in range(1, order):
            assert w @ c ** q == pytest.approx(1.0 / (q + 1), abs=1e-14)
        assert w @ a @ c == pytest.approx(1.0 / 6, abs=1e-14)
        assert w @ a @ a @ c == pytest.approx(1.0 / 24, abs=1e-14)
    assert b @ a @ c ** 3 == pytest.approx(1.0 / 20, abs=1e-14)
    assert b @ (a @ c) ** 2 == pytest.approx(1.0 / 20, abs=1e-14)
    assert b @ a @ a @ a @ c == pytest.approx(1.0 / 120, abs=1e-14)
    assert e[6] == pytest.approx(-1.0 / 40, abs=1e-17) and np.abs(e).max() > 1e-3
