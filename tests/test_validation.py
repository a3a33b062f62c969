"""Argument checks of llg_create, run on the host: every invalid problem or
option is rejected with LLG_EINVAL and a message before any device work (so
these run without a GPU), and the context returned with the error can be
destroyed without one."""
import math

import pytest

import workloads as W

N = 40


def _spectral():
    return W.random_small(12, 8, 1, seed=1, nsteps=N, objective=W.J_SPECTRAL, freqs=(8e9,), n_from=5).problem


def _curve():
    return W.random_small(12, 8, 1, seed=1, nsteps=N, objective=W.J_CURVE, comp=0, sample_steps=(10, 20),
                          sample_targets=(0.5, 0.6), sample_weights=(1.0, 1.0)).problem


def _base():
    return W.random_small(12, 8, 1, seed=1, nsteps=N).problem


BAD_PROBLEMS = {
    "nx not a multiple of 4": lambda: _base().replace(nx=6),
    "ny beyond the column FFT": lambda: _base().replace(ny=600),
    "nz beyond 8 layers": lambda: _base().replace(nz=9),
    "non-positive cell": lambda: _base().replace(dx=0.0),
    "unknown objective": lambda: _base().replace(objective=7),
    "port exponent": lambda: _base().replace(power=3),
    "spectral without frequencies": lambda: _spectral().replace(freqs=()),
    "spectral with 9 frequencies": lambda: _spectral().replace(freqs=tuple(1e9 * (k + 1) for k in range(9))),
    "spectral window at step 0": lambda: _spectral().replace(n_from=0),
    "spectral NaN frequency": lambda: _spectral().replace(freqs=(math.nan,)),
    "curve without samples": lambda: _curve().replace(sample_steps=(), sample_targets=(), sample_weights=()),
    "curve samples out of order": lambda: _curve().replace(sample_steps=(20, 10)),
    "curve sample beyond nsteps": lambda: _curve().replace(sample_steps=(10, N + 1)),
    "curve NaN weight": lambda: _curve().replace(sample_weights=(1.0, math.nan)),
    "drive table with inf": lambda: _base().replace(drive=(0.0,) * (3 * N) + (math.inf,) * 3),
}


@pytest.fixture(scope="module")
def lib():
    from paper_2411_19109_gb300 import load
    return load()


@pytest.mark.parametrize("case", sorted(BAD_PROBLEMS))
def test_invalid_problem_is_rejected_on_the_host(lib, case):
    from paper_2411_19109_gb300.llg import LLG_EINVAL, LLGError, llg_create
    with pytest.raises(LLGError) as e:
        llg_create([BAD_PROBLEMS[case]()])
    assert e.value.status == LLG_EINVAL and str(e.value).split(':', 1)[1].strip()


def test_instances_must_share_the_time_grid(lib):
    from paper_2411_19109_gb300.llg import LLG_EINVAL, LLGError, llg_create
    with pytest.raises(LLGError) as e:
        llg_create([_base(), _base().replace(nsteps=N + 1)])
    assert e.value.status == LLG_EINVAL


@pytest.mark.parametrize("kw", [dict(integrator=5), dict(integrator=1, rtol=0.0), dict(integrator=1, atol=-1.0),
                                dict(integrator=1, rtol=math.inf)])
def test_invalid_integrator_options_are_rejected(lib, kw):
    from paper_2411_19109_gb300.llg import LLG_EINVAL, LLGError, llg_create
    with pytest.raises(LLGError) as e:
        llg_create([W.random_small(12, 8, 1, nsteps=N, objective=W.J_ENERGY_AREA).problem], **kw)
    assert e.value.status == LLG_EINVAL


@pytest.mark.parametrize("p", [_base, _spectral, _curve])
def test_adaptive_integrator_needs_the_terminal_objective(lib, p):
    from paper_2411_19109_gb300.llg import LLG_EINVAL, LLGError, llg_create
    with pytest.raises(LLGError) as e:
        llg_create([p()], integrator=1, rtol=1e-5, atol=1e-8)
    assert e.value.status == LLG_EINVAL


def _wide(nx, nz=1, ny=8):
    return W.random_small(12, 8, 1, seed=1, nsteps=N).problem.replace(nx=nx, ny=ny, nz=nz)


@pytest.mark.parametrize("nx", [784, 1024])
def test_fp64_rows_wider_than_the_adjoint_tile_are_rejected(lib, nx):
    """FP64 adjoint row tile: 3840 exchange slots x 16 B + 7 arrays x 3 rows x nx x 8 B
    + the W_2048 table (32 KB) exceeds 220 KB once nx > 780."""
    from paper_2411_19109_gb300.llg import LLG_EINVAL, LLGError, llg_create
    with pytest.raises(LLGError) as e:
        llg_create([_wide(nx)], precision=1)
    assert e.value.status == LLG_EINVAL and "row tile" in str(e.value)


@pytest.mark.parametrize("nx,precision", [(780, 1), (1024, 0)])
def test_widest_supported_rows_pass_the_size_checks(lib, nx, precision):
    """Accepted by every host check: what follows is device work, so without a
    GPU the call fails later, with a status other than LLG_EINVAL."""
    import torch
    from paper_2411_19109_gb300.llg import LLG_EINVAL, LLGError, llg_create
    if torch.cuda.is_available():
        pytest.skip("would allocate on the device")
    with pytest.raises(LLGError) as e:
        llg_create([_wide(nx)], precision=precision)
    assert e.value.status != LLG_EINVAL


def test_fp64_3d_column_tile_limit_is_reported_as_a_column_tile(lib):
    from paper_2411_19109_gb300.llg import LLG_EINVAL, LLGError, llg_create
    with pytest.raises(LLGError) as e:
        llg_create([_wide(16, nz=4, ny=512)], precision=1)
    assert e.value.status == LLG_EINVAL and "column tile" in str(e.value)
