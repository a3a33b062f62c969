"""Helpers shared by the GPU parity tests: run instances through the C ABI
(via the ctypes binding) and through the FP64 oracle on the same seeded
inputs."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, float).ravel()
    b = np.asarray(b, float).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_solver(instances, precision="fp32", **kw):
    from paper_2411_19109_gb300 import Solver
    return Solver([i.problem for i in instances], precision=precision, **kw)


def gpu_run(instances, precision="fp32", adjoint=True, want_dm0=False, **kw):
    """Returns dict with J, mT, dphi (lists of numpy arrays per instance)."""
    s = gpu_solver(instances, precision, **kw)
    try:
        phi = s.pack_scalar([i.phi for i in instances])
        m0 = s.pack_vector([i.m0 for i in instances])
        J, mT = s.forward(phi, m0, want_mT=True)
        out = {"J": J, "mT": [x.double().cpu().numpy() for x in s.unpack_vector(mT)]}
        if adjoint:
            g, dm0 = s.adjoint(want_dm0=want_dm0)
            out["dphi"] = [x.double().cpu().numpy() for x in s.unpack_scalar(g)]
            if want_dm0:
                out["dm0"] = [x.double().cpu().numpy() for x in s.unpack_vector(dm0)]
        out["launches"] = s.launch_count()
        out["bytes"], out["ms"] = s.query()
        return out
    finally:
        s.close()


def oracle_run(inst, adjoint=True):
    from oracle import llg
    model = llg.Model(inst.problem, inst.phi)
    J, mN, traj = model.forward(inst.m0, keep=adjoint)
    out = {"J": J, "mT": mN}
    if adjoint:
        dphi, dm0, _ = model.adjoint(inst.m0, traj)
        out["dphi"] = dphi
        out["dm0"] = dm0
    return out
