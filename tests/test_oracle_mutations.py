"""The oracle's pins catch plausible mistakes: each case plants one mistake (a sign, a
dropped term, a wrong coefficient, a conjugated transform) in an in-memory copy of the
oracle on the CPU and requires at least one pin of tests/test_oracle_pins.py or
tests/test_oracle_adjoint.py to fail against it."""
import functools
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
    "L_- coupling sign": ("Lm = Lh - inv_r2 * I + 2.0 * mm * inv_r2 * I", "Lm = Lh - inv_r2 * I - 2.0 * mm * inv_r2 * I"),
    "m_p dropped from m m_p": ("self.mm = prm.m_p * m.astype(np.float64)", "self.mm = m.astype(np.float64)"),
    "H_z takes the 1/r^2 term": ('("Hz", Lh)):', '("Hz", Lh - inv_r2 * I)):'),
    "no row interchange": ("p = c + np.argmax(np.abs(A[c:last + 1, c]), axis=0)",
                           "p = np.full(A.shape[-1], c)"),
    "back substitution over ku super-diagonals": (
        "        hi = min(i + kl + ku, N - 1) + 1\n        s = B[i]",
        "        hi = min(i + ku, N - 1) + 1\n        s = B[i]"),
    "k = -|k| solved with the k = +|k| right-hand side": ("bp, bm = b[:, K:], b[:, K::-1]", "bp, bm = b[:, K:], b[:, K:]"),
    "adjoint transposed solve": ("return solve_modes(ops, np.swapaxes(A, -1, -2), rhs)", "return solve_modes(ops, A, rhs)"),
    "adjoint of theta-derivative": ("+ np.conj(im) * _to_physical_T(ops, bar[(\"t\", c)])", "+ im * _to_physical_T(ops, bar[(\"t\", c)])"),
}


def _calls(module, names):
    """Every pin as a zero-argument call; a parametrised pin gives one call per value."""
    out = []
    for n in names:
        f = getattr(module, n)
        marks = [m for m in getattr(f, "pytestmark", []) if m.name == "parametrize"]
        if not marks:
            out.append(f)
            continue
        (argname, values), = [m.args for m in marks]
        out += [functools.partial(f, **{argname: v}) for v in values]
    return out


FAST_PINS = _calls(PINS, [n for n in dir(PINS) if n.startswith("test_") and n !=
                          "test_taylor_vortex_onset_bracket"] + ["test_taylor_vortex_onset_bracket"])
ADJ_PINS = _calls(ADJ, [n for n in dir(ADJ) if n.startswith("test_")])


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
        except TypeError:
            raise           # a pin called with the wrong arguments proves nothing
        except Exception:
            return          # caught
    pytest.fail(f"no pin caught the planted mistake: {name}")
