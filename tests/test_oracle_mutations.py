"""The oracle's pins catch plausible mistakes: each case plants one mistake (a sign, a
dropped term, a wrong coefficient, a conjugated transform) in an in-memory copy of the
oracle on the CPU and requires at least one pin of tests/test_oracle_pins.py or
tests/test_oracle_adjoint.py to fail against it."""
import os
import types

import pytest

import oracle
import tests.test_oracle_adjoint as ADJ
import tests.test_oracle_pins as PINS

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "tc_oracle.py")).read()

MUTATIONS = {
    "curvature N_theta sign": ("Nt = adv(ut_r, ut_t, ut_z) + ut * ur / r", "Nt = adv(ut_r, ut_t, ut_z) - ut * ur / r"),
    "centripetal sign": ("Nr = adv(ur_r, ur_t, ur_z) - ut * ut / r", "Nr = adv(ur_r, ur_t, ur_z) + ut * ut / r"),
    "drop (1/r) d_r in Laplacian": ("base = D2 + inv_r * D1", "base = D2"),
    "L_+ coupling sign": ("Lp = Lh - inv_r2 * I - 2.0 * mm * inv_r2 * I", "Lp = Lh - inv_r2 * I + 2.0 * mm * inv_r2 * I"),
    "gradient +- sign": ("return np.stack([d - t, d + t,", "return np.stack([d + t, d - t,"),
    "drop Laplacian in Neumann rows": (
        "+ 2.0 * vector_laplacian_r(ops, u) - vector_laplacian_r(ops, u_prev)", "+ 0.0"),
    "pressure update coefficient": ("p_new = p_star + 3.0 * phi / (2.0 * dt)", "p_new = p_star + phi / dt"),
    "AB2 extrapolation dropped": ("rhs = (4.0 * u - u_prev) / (2.0 * dt) - NN - gp", "rhs = (4.0 * u - u_prev) / (2.0 * dt) - N - gp"),
    "divergence theta term": ("ops.mm[None, :, None] * (vp - vm) / (2.0 * r)", "ops.mm[None, :, None] * (vp + vm) / (2.0 * r)"),
    "inverse theta transform sign": ("self.G = _unit_roots(Pt, np.outer(a, m), +1)", "self.G = _unit_roots(Pt, np.outer(a, m), -1)"),
    "start-up extrapolation": ("u_m1 = u0 - 1.5 * (u_e - u0)", "u_m1 = u0"),
    "adjoint transposed solve": ("return solve_modes(ops, np.swapaxes(A, -1, -2), rhs)", "return solve_modes(ops, A, rhs)"),
    "adjoint of theta-derivative": ("+ np.conj(im) * _to_physical_T(ops, bar[(\"t\", c)])", "+ im * _to_physical_T(ops, bar[(\"t\", c)])"),
}

FAST_PINS = [getattr(PINS, n) for n in dir(PINS) if n.startswith("test_") and n not in
             ("test_taylor_vortex_onset_bracket",)] + [PINS.test_taylor_vortex_onset_bracket]
ADJ_PINS = [getattr(ADJ, n) for n in dir(ADJ) if n.startswith("test_")]


def _mutant(old, new):
    assert SRC.count(old) >= 1, old
    mod = types.ModuleType("oracle_mutant")
    exec(compile(SRC.replace(old, new), "tc_oracle_mutant.py", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_a_pin_fails_for_each_planted_mistake(name, monkeypatch):
    mod = _mutant(*MUTATIONS[name])
    monkeypatch.setattr(PINS, "O", mod)
    monkeypatch.setattr(ADJ, "O", mod)
    for pin in ADJ_PINS + FAST_PINS:
        try:
            pin()
        except Exception:
            return          # caught
    pytest.fail(f"no pin caught the planted mistake: {name}")
