"""tc_nonlinear_noalloc: the nonlinear term for callers that may not allocate device memory.

Some callers cannot call cudaMalloc (a real-time host loop, a plug-in whose host framework
owns all device memory, a caller with no workspace to hand over).  The entry point keeps its
staging in a static 80 MiB device array instead.  This file is collected last so that a run
stopping at the first failure has already run every other test.  It checks, through the C
ABI, two calls in a row against tc_nonlinear with a caller workspace (FP64 plans, and mixed
plans after another plan's call has left different data in the array), that a call allocates
nothing, and the size and host-plan rejections.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1311_2481_gb300 import build as B  # noqa: E402
from paper_1311_2481_gb300 import inputs as I  # noqa: E402
from paper_1311_2481_gb300 import tc  # noqa: E402

B.build()
LZ = 2 * math.pi / 3.16


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("cfg", [
    dict(N_r=32, M=8, K=16, Re_i=50.0, dt=1e-3),      # small parity configuration
    dict(N_r=64, M=32, K=64, Re_i=1000.0, dt=5e-4),   # benchmark size (74 MiB of staging)
])
def test_noalloc_matches_workspace_path_on_two_calls(cfg):
    lib = tc.load_library()
    plan = tc.Plan(m_p=1, eta=0.5, Re_o=0.0, L_z=LZ, **cfg)
    r = plan.nodes()
    outs = []
    for seed in (42, 43):
        u = torch.from_numpy(I.initial_state(r, cfg["M"], cfg["K"], 1, LZ, 0.5, cfg["Re_i"], 0.0,
                                             kind="box", amp=1e-2, seed=seed)).cuda()
        ref = plan.nonlinear(u)
        got = torch.full_like(u, float("nan"))
        st = lib.tc_nonlinear_noalloc(plan.handle, ctypes.c_void_p(u.data_ptr()),
                                      ctypes.c_void_p(got.data_ptr()), _stream())
        assert st == tc.TC_OK, lib.tc_plan_last_error(plan.handle)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
        outs.append(a)
    assert not np.allclose(outs[0], outs[1])   # the second call did not reuse the first result


@pytest.mark.parametrize("no_adjoint", [False, True])
def test_noalloc_mixed_plan_after_another_layout(no_adjoint):
    """A TC_MIXED plan (FP32 staging lines and the FP32 split of u, with and without the
    adjoint regions after them) through the static array right after a call of an FP64 plan
    of another size has left its own data there, on two calls in a row; the second call
    allocates nothing (the device's free memory is unchanged across it)."""
    lib = tc.load_library()
    other = tc.Plan(64, 32, 64, 1, 0.5, 1000.0, 0.0, LZ, 5e-4)
    ro = other.nodes()
    uo = torch.from_numpy(I.initial_state(ro, 32, 64, 1, LZ, 0.5, 1000.0, 0.0, kind="box", amp=1e-2,
                                          seed=7)).cuda()
    No = torch.empty_like(uo)
    assert lib.tc_nonlinear_noalloc(other.handle, ctypes.c_void_p(uo.data_ptr()),
                                    ctypes.c_void_p(No.data_ptr()), _stream()) == tc.TC_OK
    torch.cuda.synchronize()
    plan = tc.Plan(32, 12, 24, 1, 0.5, 200.0, 0.0, LZ, 1e-3, precision=tc.TC_MIXED, no_adjoint=no_adjoint)
    r = plan.nodes()
    for seed in (42, 43):
        u = torch.from_numpy(I.initial_state(r, 12, 24, 1, LZ, 0.5, 200.0, 0.0, kind="broadband", amp=1e-2,
                                             seed=seed)).cuda()
        ref = plan.nonlinear(u)
        got = torch.full_like(u, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = lib.tc_nonlinear_noalloc(plan.handle, ctypes.c_void_p(u.data_ptr()),
                                      ctypes.c_void_p(got.data_ptr()), _stream())
        torch.cuda.synchronize()
        assert st == tc.TC_OK, lib.tc_plan_last_error(plan.handle)
        assert torch.cuda.mem_get_info()[0] == free0
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_noalloc_rejects_host_plans_with_a_message():
    lib = tc.load_library()
    plan = tc.Plan(16, 4, 4, 1, 0.5, 50.0, 0.0, LZ, 1e-3, host_only=True)
    assert lib.tc_nonlinear_noalloc(plan.handle, None, None, None) == tc.TC_ERR_STATE
    assert b"host-only" in lib.tc_plan_last_error(plan.handle)


def test_noalloc_rejects_plans_beyond_the_static_scratch():
    lib = tc.load_library()
    plan = tc.Plan(128, 64, 128, 1, 0.5, 100.0, 0.0, LZ, 1e-4)   # needs ~0.6 GB of staging
    u = torch.zeros(plan.vector_shape(), dtype=torch.complex128, device="cuda")
    N = torch.zeros_like(u)
    st = lib.tc_nonlinear_noalloc(plan.handle, ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(N.data_ptr()), _stream())
    assert st == tc.TC_ERR_ARG
    assert b"static scratch" in lib.tc_plan_last_error(plan.handle)


def test_noalloc_fits_with_fewer_staged_rows():
    """The same FP64 plan with its transforms staged 16 radial rows at a time needs 77 MB of
    staging, fits the static array, and gives the workspace path's result."""
    lib = tc.load_library()
    plan = tc.Plan(128, 64, 128, 1, 0.5, 100.0, 0.0, LZ, 1e-4, stage_rows=16)
    r = plan.nodes()
    u = torch.from_numpy(I.initial_state(r, 64, 128, 1, LZ, 0.5, 100.0, 0.0, kind="box", amp=1e-2,
                                         seed=3)).cuda()
    ref = plan.nonlinear(u)
    got = torch.full_like(u, float("nan"))
    st = lib.tc_nonlinear_noalloc(plan.handle, ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(got.data_ptr()), _stream())
    assert st == tc.TC_OK, lib.tc_plan_last_error(plan.handle)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
