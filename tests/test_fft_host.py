"""The register FFT passes of the CUDA path (csrc/regfft.cuh), compiled for the
host and driven through the same Stockham schedule as the kernels
(tests/host_fft_passes.cu): every length 8..2048 with 8 elements per thread
and 16..2048 with 16, FP32 and FP64, forward and inverse, with and without the
W^4k table.  Checked against a direct DFT in long double, and every pass must
scatter its outputs to a permutation of the sequence (no two lanes write one
shared-memory slot).  Covers lengths the GPU tests do not reach (rows of
1024 and 2048 complex elements).  The double-float precision (hi + lo FP32
pairs, the adjoint's frequency-domain option) runs the same passes and must
reach the few 2^-48 its arithmetic promises."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cases(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path_factory.mktemp("fft") / "fft_passes"
    subprocess.run([nvcc, "-std=c++17", "-O1", "-DLLG_HOST_COUNT_OPS", "-I", os.path.join(ROOT, "paper_2411_19109_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_fft_passes.cu"), "-o", str(exe)],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=600).stdout
    rows, half, ops = [], [], []
    for line in out.split("\n"):
        if line.startswith("half "):
            _, prec, L, d, ok = line.split()
            half.append((prec, int(L), int(d), int(ok)))
        elif line.startswith("ops "):
            _, L, d, h, n = line.split()
            ops.append((int(L), int(d), int(h), int(n)))
        elif line.strip():
            prec, w, L, d, t4, err, perm = line.split()
            rows.append((prec, int(w), int(L), int(d), int(t4), float(err), int(perm)))
    return rows, half, ops


@pytest.fixture(scope="module")
def passes(cases):
    return cases[0]


def test_every_length_and_width_is_covered(passes):
    got = {(p, w, L, d) for p, w, L, d, *_ in passes}
    for p in ("f32", "f64", "df"):
        for d in (-1, 1):
            for k in range(3, 12):
                assert (p, 8, 2 ** k, d) in got
            for k in range(4, 12):
                assert (p, 16, 2 ** k, d) in got


def test_every_pass_scatters_to_a_permutation(passes):
    assert all(c[6] == 1 for c in passes)


def test_passes_compute_the_dft(passes):
    # FP32: a few ulp per pass (the twiddle powers are formed by products);
    # FP64: rounding only; double-float: a few 2^-48 = 3.6e-15 per pass
    bound = {"f32": 5e-7, "f64": 1e-15, "df": 2e-14}
    for prec, w, L, d, t4, err, _ in passes:
        assert err < bound[prec], (prec, w, L, d, t4, err)


def test_half_input_first_pass_equals_the_full_pass(cases):
    """The forward transforms of zero-padded data (column pass, row
    transforms) run their double-float first pass without the zero upper
    half of the inputs; every length and precision must give the full
    pass's values and destinations."""
    half = cases[1]
    assert {(p, L) for p, L, d, _ in half if d == -1} == {(p, 2 ** k) for p in ("f32", "f64", "df")
                                                         for k in range(3, 12)}
    assert all(ok == 1 for *_, ok in half), [h for h in half if h[3] != 1]


def test_operation_model_counts_the_transforms(cases):
    """The ALU roofline of the double-float kernels divides an operation
    model (bench._df_fft_ops) by the measured time; the host build counts
    the FP32 operations the transform code performs (every compensated sum,
    product and fused multiply-add of dfloat.cuh), which must equal the model
    at every length, forward (full and half-input first pass) and inverse."""
    import bench
    ops = cases[2]
    assert {L for L, *_ in ops} == {2 ** k for k in range(3, 12)}
    for L, d, h, n in ops:
        assert n == bench._df_fft_ops(L, half_in=bool(h)), (L, d, h, n, bench._df_fft_ops(L, half_in=bool(h)))
