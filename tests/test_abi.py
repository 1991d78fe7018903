"""C-ABI checks that need no GPU: the library loads, exports every symbol include/tc.h
declares, validates arguments on the host, and its host plan (nodes, FD weights) agrees
with the oracle's independent construction."""
import math
import os
import re

import numpy as np
import pytest

from paper_1311_2481_gb300 import build as B
from paper_1311_2481_gb300 import tc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return tc.load_library()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "tc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(tc_[a-z_0-9]+)\s*\(", hdr))
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(tc.SYMBOLS)


def test_argument_validation_before_any_launch(lib):
    L = 2 * math.pi / 3.16
    bad = [
        dict(N_r=8, M=8, K=16),            # N_r < fd_order + 1
        dict(N_r=32, M=0, K=16),
        dict(N_r=32, M=8, K=16, eta=1.5),
        dict(N_r=32, M=8, K=16, dt=-1.0),
        dict(N_r=32, M=5, K=16),           # P_theta = 15 is not 2^a 3^b
    ]
    for kw in bad:
        args = dict(N_r=32, M=8, K=16, m_p=1, eta=0.5, Re_i=50.0, Re_o=0.0, L_z=L, dt=1e-3)
        args.update(kw)
        with pytest.raises(tc.TCError) as e:
            tc.Plan(**args, host_only=True)
        assert e.value.status == tc.TC_ERR_ARG
    with pytest.raises(tc.TCError):
        tc.Plan(32, 8, 16, 1, 0.5, 50.0, 0.0, L, 1e-3, P_theta=16, host_only=True)   # < 2M+1


def test_host_only_plan_rejects_compute_calls(lib):
    p = tc.Plan(16, 4, 4, 1, 0.5, 50.0, 0.0, 2.0, 1e-3, host_only=True)
    st = lib.tc_nonlinear(p.handle, None, None, None, None)
    assert st == tc.TC_ERR_STATE
    st = lib.tc_step(p.handle, None, 1, None, None)
    assert st == tc.TC_ERR_STATE
    assert p.ws_bytes > 0
    assert lib.tc_status_string(tc.TC_ERR_NONFINITE).decode() == "non-finite value in state"


def test_host_plan_matches_oracle_nodes_and_weights(lib):
    import oracle as O
    for (N, alpha) in ((32, 0.5), (45, 1.0), (24, 0.0)):
        L = 2 * math.pi / 3.16
        p = tc.Plan(N, 4, 4, 1, 0.5, 50.0, 0.0, L, 1e-3, alpha=alpha, host_only=True)
        ops = O.Operators(O.Params(N, 4, 4, 1, 0.5, 50.0, 0.0, L, 1e-3, alpha=alpha))
        np.testing.assert_array_max_ulp(p.nodes(), ops.r, maxulp=1)
        for deriv, ref in ((1, ops.D1), (2, ops.D2)):
            w, c = p.fd_weights(deriv)
            D = np.zeros((N, N))
            for j in range(N):
                D[j, c[j]:c[j] + 9] = w[j]
            assert np.abs(D - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("N", [15, 16, 25, 48, 96, 128])
def test_host_factors_solve_the_mode_systems(lib, N):
    """The stored pivoted banded LU factors of every system (Sec. 3.2: Eq. pressure, Eq. vel,
    Eq. correction) and their two-partition form (the diagonal blocks' own LU factors, the
    spikes and the inverse 8 x 8 reduced matrix) solve the oracle's mode matrices: against
    the oracle's own banded elimination, on random right-hand sides.  N_r = 15 has no
    two-partition form."""
    import oracle as O
    L = 2 * math.pi / 3.16
    cfg = (N, 6, 8, 1, 0.5, 300.0, 0.0, L, 1e-3)
    p = tc.Plan(*cfg, host_only=True)
    ops = O.Operators(O.Params(*cfg))
    rng = np.random.default_rng(3)
    names = {tc.TC_P_STAR: "P", tc.TC_U_PLUS: "Hp", tc.TC_U_MINUS: "Hm", tc.TC_U_Z: "Hz", tc.TC_PHI: "P"}
    worst = 0.0
    for which, name in names.items():
        for (m, ka) in ((0, 0), (0, 3), (1, 0), (6, 8), (3, 5)):
            A = ops.mats[name][m, ka]
            b = rng.standard_normal(N)
            ref = O.gauss_banded(A, b[:, None])[:, 0]
            # two backward-stable pivoted eliminations in different rounding order differ by
            # at most about eps * cond(A); the bound asked for is 5e-4 of that
            tol = 1e-13 + 1e-19 * np.linalg.cond(A)
            for parts in (1, 2):
                if parts == 2 and N < 16:
                    with pytest.raises(tc.TCError) as e:
                        p.solve_host(which, m, ka, b, parts)
                    assert e.value.status == tc.TC_ERR_STATE
                    continue
                x = p.solve_host(which, m, ka, b, parts)
                err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
                worst = max(worst, err / tol)
                assert err <= tol, (which, m, ka, parts, err, tol)
    print("worst fraction of the bound", worst)


def test_plan_options_validated(lib):
    """Out-of-range launch options are rejected at plan creation; pc_partitions = 1 leaves
    the plan without the two-partition form (its host solve then reports TC_ERR_STATE)."""
    L = 2 * math.pi / 3.16
    args = (24, 4, 4, 1, 0.5, 50.0, 0.0, L, 1e-3)
    for kw in (dict(pc_partitions=3), dict(pc_partitions=-1), dict(pc_split=2), dict(theta_variant=5),
               dict(pc_modes=33)):
        with pytest.raises(tc.TCError) as e:
            tc.Plan(*args, host_only=True, **kw)
        assert e.value.status == tc.TC_ERR_ARG, kw
    b = np.linspace(0.0, 1.0, 24)
    p2 = tc.Plan(*args, host_only=True)
    p1 = tc.Plan(*args, host_only=True, pc_partitions=1)
    assert np.allclose(p2.solve_host(tc.TC_U_Z, 2, 3, b, 2), p1.solve_host(tc.TC_U_Z, 2, 3, b, 1), rtol=1e-12)
    with pytest.raises(tc.TCError) as e:
        p1.solve_host(tc.TC_U_Z, 2, 3, b, 2)
    assert e.value.status == tc.TC_ERR_STATE


def test_plan_set_on_host_plan(lib):
    """tc_plan_set rebuilds what depends on the setting (here the nodes of Eq. nodeDist and the
    factors), rejects unknown keys and out-of-range values without changing the plan, and a
    rebuilt plan equals one created with the setting."""
    L = 2 * math.pi / 3.16
    args = (24, 4, 4, 1, 0.5, 50.0, 0.0, L, 1e-3)
    a = tc.Plan(*args, host_only=True)
    b = tc.Plan(*args, host_only=True, alpha=0.9)
    r0 = a.nodes()
    a.set(tc.TC_SET_ALPHA, 0.9)
    assert np.array_equal(a.nodes(), b.nodes()) and not np.array_equal(a.nodes(), r0)
    rhs = np.linspace(-1.0, 2.0, 24)
    assert np.array_equal(a.solve_host(tc.TC_U_PLUS, 2, 3, rhs), b.solve_host(tc.TC_U_PLUS, 2, 3, rhs))
    for key, value in ((99, 1.0), (tc.TC_SET_P_THETA, 7.0), (tc.TC_SET_P_THETA, 12.5),
                       (tc.TC_SET_PRECISION, 5.0), (tc.TC_SET_ALPHA, 2.0), (tc.TC_SET_PC_SPLIT, 3.0)):
        with pytest.raises(tc.TCError) as e:
            a.set(key, value)
        assert e.value.status == tc.TC_ERR_ARG, (key, value)
    assert np.array_equal(a.nodes(), b.nodes())
    ws0 = a.ws_bytes
    a.set(tc.TC_SET_NO_ADJOINT, 1)
    assert a.ws_bytes < ws0
    # staging by radial slab: fewer rows per slab, less workspace; negative rows are refused
    ws1 = a.ws_bytes
    a.set(tc.TC_SET_STAGE_ROWS, 5)
    assert a.ws_bytes < ws1
    assert a.ws_bytes == tc.Plan(*args, host_only=True, alpha=0.9, no_adjoint=True, stage_rows=5).ws_bytes
    for key, value in ((tc.TC_SET_STAGE_ROWS, -1.0), (tc.TC_SET_MEAN_FP32, 2.0)):
        with pytest.raises(tc.TCError) as e:
            a.set(key, value)
        assert e.value.status == tc.TC_ERR_ARG, (key, value)
    a.set(tc.TC_SET_MEAN_FP32, 1)   # accepted on any plan; only the mixed form reads it


def test_stage_rows_workspace_layout():
    """The FP64 staging of a plan holds 12 line sets of stage_rows radial rows (21 with the
    adjoint); all rows while they fit 4 GiB.  A mixed plan's FP32 forward staging keeps all
    rows whatever stage_rows is."""
    L = 2 * math.pi / 3.16
    args = (40, 8, 16, 1, 0.5, 50.0, 0.0, L, 1e-3)
    line = 9 * 48 * 16                          # (M+1) P_z complex128 values of one row
    full = tc.Plan(*args, host_only=True, no_adjoint=True).ws_bytes
    part = tc.Plan(*args, host_only=True, no_adjoint=True, stage_rows=10).ws_bytes
    assert full - part >= 12 * 30 * line         # 12 line sets of 30 rows fewer (256-byte rounding aside)
    assert full - part < 12 * 30 * line + 4 * 256
    m_full = tc.Plan(*args, host_only=True, no_adjoint=True, precision=tc.TC_MIXED).ws_bytes
    m_part = tc.Plan(*args, host_only=True, no_adjoint=True, precision=tc.TC_MIXED, stage_rows=10).ws_bytes
    assert m_full == m_part
