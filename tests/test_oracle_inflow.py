"""Pins of the oracle's reservoir inflow state (Sec. 4, the nozzle inlet
boundary condition: the reservoir's entropy and the enthalpy balance with the
reservoir at rest).

Each check is a consequence of the two printed conditions worked out by hand,
not a retyping of the formulas: substitution into both conditions, the case
of no pressure drop, and a closed form for a Mach-3 inflow.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
@pytest.mark.parametrize("ratio", [0.9, 0.3, 0.027, 1e-3])
def test_inflow_state_satisfies_both_conditions(oracle_lib, gamma, ratio):
    P_res, rho_res = 36.9, 13.1
    P = ratio * P_res
    rho, u = oracle.inflow_state(gamma, P_res, rho_res, P)
    # the reservoir's entropy
    assert abs(P / rho ** gamma - P_res / rho_res ** gamma) <= 1e-13 * P_res / rho_res ** gamma
    # the enthalpy balance, u_res = 0
    c2, c2r = gamma * P / rho, gamma * P_res / rho_res
    assert abs(0.5 * u * u + c2 / (gamma - 1.0) - c2r / (gamma - 1.0)) <= 1e-13 * c2r / (gamma - 1.0)
    assert u > 0.0


def test_no_pressure_drop_no_inflow(oracle_lib):
    rho, u = oracle.inflow_state(1.4, 2.0, 0.5, 2.0)
    assert rho == 0.5 and u == 0.0
    rho, u = oracle.inflow_state(1.4, 2.0, 0.5, 3.0)     # above the reservoir's: no inflow
    assert u == 0.0


def test_mach_three_inflow(oracle_lib):
    # Mach M inflow from rest: c_res^2 / c_inf^2 = 1 + (gamma - 1) M^2 / 2 = 2.8 for
    # gamma = 1.4, M = 3, and along the isentrope P_inf / P_res = (c_inf / c_res)^(2 gamma / (gamma - 1))
    # = (1 / 2.8)^3.5
    g = 1.4
    rho, u = oracle.inflow_state(g, 1.0, 1.0, 2.8 ** -3.5)
    c = np.sqrt(g * 2.8 ** -3.5 / rho)
    assert abs(u / c - 3.0) < 1e-12
    assert abs(rho - 2.8 ** -2.5) < 1e-14         # rho / rho_res = (P / P_res)^(1/gamma) = 2.8^-2.5
