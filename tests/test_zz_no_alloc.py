"""llg_field_noalloc, the allocation-free field evaluation, against llg_field.

Some callers cannot allocate device memory where they evaluate a field (a
framework that owns all device memory through its own allocator, a loop
where cudaMalloc's synchronisation would stall other streams).
llg_field_noalloc serves them from a fixed scratch array in the library; it
must give the same field as the context-based llg_field.

Calls in a row with different grids and modes check that a call does not
depend on what the previous one left in the shared scratch, and a repeated
grid that the spectrum kept from the previous call is still right.  Grids at
the scratch's bound (128 x 128) and with 128-point columns (64 x 64) compare
its 8-element column kernel with the 16-element one llg_field takes there.
This file is collected last (test_zz_*) so that a run stopping at its first
failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_solver, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 2e-6   # the FP32 field-parity tolerance of test_gpu_parity


def _reference_field(inst, t, demag_only):
    s = gpu_solver([inst], "fp32")
    try:
        phi = s.pack_scalar([inst.phi])
        m = s.pack_vector([inst.m0])
        return s.field(phi, m, t, demag_only=demag_only).cpu().numpy()
    finally:
        s.close()


def _noalloc_field(inst, t, demag_only):
    from paper_2411_19109_gb300 import llg_field_noalloc
    phi = torch.as_tensor(inst.phi.reshape(-1), dtype=torch.float32).cuda()
    m = torch.as_tensor(inst.m0.reshape(-1), dtype=torch.float32).cuda()
    B = torch.empty_like(m)
    stream = torch.cuda.current_stream()
    llg_field_noalloc(inst.problem, phi.data_ptr(), m.data_ptr(), t, demag_only, B.data_ptr(),
                      stream.cuda_stream)
    torch.cuda.synchronize()
    return B.cpu().numpy()


def test_noalloc_field_matches_llg_field_twice():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    first = W.random_small(32, 20, 1, seed=21)
    second = W.random_small(16, 12, 1, seed=22)
    a = _noalloc_field(first, 2.5e-11, False)
    assert rel_l2(a, _reference_field(first, 2.5e-11, False)) < TOL
    b = _noalloc_field(second, 0.0, True)
    assert rel_l2(b, _reference_field(second, 0.0, True)) < TOL
    assert np.isfinite(a).all() and np.isfinite(b).all()


def test_noalloc_field_at_the_scratch_bound():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    for shape, t, demag_only in (((128, 128), 1.0e-11, False), ((64, 64), 0.0, True), ((64, 64), 3.0e-11, False),
                                 ((128, 128), 0.0, True)):
        inst = W.random_small(*shape, 1, seed=shape[0] + int(demag_only))
        a = _noalloc_field(inst, t, demag_only)
        assert rel_l2(a, _reference_field(inst, t, demag_only)) < TOL, shape


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2411_19109_gb300 import LLGError
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    big = W.random_small(132, 8, 1, seed=1)
    with pytest.raises(LLGError, match="fixed scratch"):
        _noalloc_field(big, 0.0, False)
