"""Failure detection without a GPU fault: the tensor-core transform's mbarrier waits are
bounded; with its tile loads withheld every CTA's first wait expires, the kernel records
WP_ERR_TIMEOUT in its status word and returns, and the CUDA context stays usable (a normal
kernel generation right after it matches the oracle and reports status 0)."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import KERNEL_TOL, f32, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_expires_with_status_and_context_survives():
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300 import _lib

    dev = torch.device("cuda")
    N, dl, R, P = 256, np.deg2rad(2.0) / 256, 512, 16
    plan = wp.Plan(N, dl, 8, 15, 3, 0.0, R, "cubic", "tf32x3")
    ws = wp.kernelgen_prepare(plan, P)
    lib = _lib.load()
    radial = torch.zeros((P, plan.geometry().k_out), dtype=torch.complex64, device=dev)
    status = ctypes.c_int32(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.wp_selftest_bounded_wait(ctypes.byref(plan.c()), P, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      ctypes.c_void_p(radial.data_ptr()), ctypes.byref(status), stream)
    assert rc == 0
    assert status.value == -6                       # WP_ERR_TIMEOUT
    assert float(torch.abs(radial).max()) == 0.0     # nothing written
    # the context is intact: the same workspace generates correct kernels
    taper = synth.gaussian_taper_samples(N, dl, R)
    planes = np.linspace(0.0, 500.0, P)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), planes,
                          supports=[5] * P, ws=ws, prepare=False)
    assert lib.wp_kernelgen_status(ctypes.byref(plan.c()), P, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                   ctypes.byref(status), stream) == 0
    assert status.value == 0
    g = o.Geometry(N, dl, 8, 15, 3, 0.0, R)
    ks = o.wkernels(g, f32(taper), planes, supports=[5] * P)
    assert rel_l2(wk.radial.cpu().numpy(), ks.radial) < KERNEL_TOL
