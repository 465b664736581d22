"""The ERK-ESDIRK time integrator of Eq. (GePUP-IMEX) (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names the additive Runge-Kutta family of Kennedy & Carpenter (ERK-ESDIRK) and a
fourth-order scheme, and leaves the coefficients to a cited appendix.  Reading: the
six-stage, fourth-order member ARK4(3)6L[2]SA of that family (explicit first stage,
gamma = a^[I]_{ss} = 1/4, stiffly accurate: b equals the last row of A^[I]), restated here
as exact rationals; the tests pin it by the order conditions of both parts and their
coupling conditions up to order four, and by fourth-order convergence of an additive
integration.
"""
from fractions import Fraction as F

import numpy as np

STAGES = 6
GAMMA = F(1, 4)

C = [F(0), F(1, 2), F(83, 250), F(31, 50), F(17, 20), F(1)]

A_E = [[F(0)] * 6 for _ in range(6)]
A_E[1][0] = F(1, 2)
A_E[2][:2] = [F(13861, 62500), F(6889, 62500)]
A_E[3][:3] = [F(-116923316275, 2393684061468), F(-2731218467317, 15368042101831),
              F(9408046702089, 11113171139209)]
A_E[4][:4] = [F(-451086348788, 2902428689909), F(-2682348792572, 7519795681897),
              F(12662868775082, 11960479115383), F(3355817975965, 11060851509271)]
A_E[5][:5] = [F(647845179188, 3216320057751), F(73281519250, 8382639484533), F(552539513391, 3454668386233),
              F(3354512671639, 8306763924573), F(4040, 17871)]

B = [F(82889, 524892), F(0), F(15625, 83664), F(69875, 102672), F(-2260, 8211), F(1, 4)]

A_I = [[F(0)] * 6 for _ in range(6)]
A_I[1][:2] = [GAMMA, GAMMA]
A_I[2][:3] = [F(8611, 62500), F(-1743, 31250), GAMMA]
A_I[3][:4] = [F(5012029, 34652500), F(-654441, 2922500), F(174375, 388108), GAMMA]
A_I[4][:5] = [F(15267082809, 155376265600), F(-71443401, 120774400), F(730878875, 902184768),
              F(2285395, 8070912), GAMMA]
A_I[5][:6] = list(B)


def tableau(dtype=float):
    """(A_E, A_I, b, c) as float arrays."""
    return (np.array(A_E, dtype=dtype), np.array(A_I, dtype=dtype), np.array(B, dtype=dtype),
            np.array(C, dtype=dtype))


def ark_step(y, t, k, f_e, f_i, solve_i):
    """One additive Runge-Kutta step of y' = f_e(t, y) + f_i(t, y), the structure of Eq.
    (GePUP-IMEX): for s = 2..6, (I - k gamma f_i) Y_s = y + k sum_j a^E_sj f_e(Y_j)
    + k sum_j a^I_sj f_i(Y_j) (j < s), solved by ``solve_i(rhs, t_s, k gamma)``; then
    y_new = Y_6 + k sum_j (b_j - a^E_6j) f_e(Y_j) (stiff accuracy: the implicit part needs
    no update)."""
    AE, AI, b, c = tableau()
    Y, FE, FI = [y], [f_e(t, y)], [f_i(t, y)]
    for s in range(1, STAGES):
        rhs = y + k * sum(AE[s, j] * FE[j] for j in range(s)) + k * sum(AI[s, j] * FI[j] for j in range(s))
        ys = solve_i(rhs, t + c[s] * k, k * float(GAMMA))
        Y.append(ys)
        FE.append(f_e(t + c[s] * k, ys))
        FI.append(f_i(t + c[s] * k, ys))
    return Y[-1] + k * sum((b[j] - AE[STAGES - 1, j]) * FE[j] for j in range(STAGES))
