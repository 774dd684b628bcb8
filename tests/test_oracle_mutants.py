"""Mutation tests of the oracle's pins (CPU only).

Each test compiles a copy of the oracle with one term of the paper's scheme
dropped or its sign flipped -- the plausible slips a transcription could
make -- and checks that the pin written for that term rejects the copy.
The committed oracle is untouched; the copies live in a temporary folder.
"""
import pytest

import oracle
from tests import oracle_runs

DT_PSIU = "double dtx = pux - s->psiux_prev[k], dty = puy - s->psiuy_prev[k];"
SOURCE = "double Q = r * cp[k] * T[k] * mdot[k];"

MUTANTS = {
    # Sec. 3.1, Eq. (eq23): the Euler derivative d_t(psi u) in the source F_i
    "dt_psiu_dropped": (DT_PSIU, "double dtx = 0.0 * (pux - s->psiux_prev[k]), dty = 0.0 * (puy - s->psiuy_prev[k]);"),
    "dt_psiu_flipped": (DT_PSIU, "double dtx = -(pux - s->psiux_prev[k]), dty = -(puy - s->psiuy_prev[k]);"),
    # Sec. 3.3, Eq. (LB_H): the source rho C_p T mdot (and its half in the H recovery)
    "source_dropped": (SOURCE, "double Q = 0.0 * (r * cp[k] * T[k] * mdot[k]);"),
    "source_flipped": (SOURCE, "double Q = -(r * cp[k] * T[k] * mdot[k]);"),
}


def _mutant(tmp_path_factory, name):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, "the mutated line must exist once in the oracle"
    return oracle.build_variant(src.replace(old, new), str(tmp_path_factory.mktemp("mutants")), name)


@pytest.mark.parametrize("name", ["dt_psiu_dropped", "dt_psiu_flipped"])
def test_translating_drop_pin_rejects_a_wrong_dt_psiu(tmp_path_factory, name):
    """The translating-drop pin (test_oracle_pins) fails without d_t(psi u)
    or with its sign flipped."""
    r = oracle_runs.translating_drop(0.1, lib=_mutant(tmp_path_factory, name))
    assert abs(r["aniso"] - 1) > 0.025, r["aniso"]


@pytest.mark.parametrize("name", ["source_dropped", "source_flipped"])
def test_temperature_origin_pin_rejects_a_wrong_enthalpy_source(tmp_path_factory, name):
    """The temperature-origin pin (test_oracle_pins) fails without the
    enthalpy source or with its sign flipped."""
    L = _mutant(tmp_path_factory, name)
    f0 = oracle_runs.shifted_layer(0.0, lib=L)["frozen"]
    f2 = oracle_runs.shifted_layer(2.0, lib=L)["frozen"]
    assert abs(f2 / f0 - 1) > 0.03, (f0, f2)
