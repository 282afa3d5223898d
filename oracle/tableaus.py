"""IMEX Butcher tableaus in the generic form of App. A, Tab. butcher_tableaus.

TEST INFRASTRUCTURE ONLY (see oracle/element.py).

Stages are numbered i = 0..s-1; stage 0 is explicit (Q_0 = Q^n), so the implicit tableau has
a zero first column and b_im[0] = 0 (Sec. 2.6). Arrays: A_ex, A_im (s x s), b_ex, b_im, c (s).

ARS(2,2,2) and ARS(3,4,3) are not printed in the paper (it cites Ascher, Ruuth and Spiteri,
1997, for IMEX-RK methods); their coefficients are those of that publication. The paper's own
tableaus (IMEX Euler, SSP2(3,3,2), SSP3(4,3,3)) are in App. A.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Tableau:
    name: str
    A_ex: np.ndarray
    b_ex: np.ndarray
    A_im: np.ndarray
    b_im: np.ndarray
    c: np.ndarray

    @property
    def s(self):
        return len(self.c)

    @property
    def fits_alg1(self):
        """Alg. 1 assumes a_{i,0}^im = b_0^im = 0 and a_{i,i}^im != 0 for i >= 1."""
        return (np.all(self.A_im[:, 0] == 0) and self.b_im[0] == 0
                and np.all(np.diag(self.A_im)[1:] != 0))


def ars222():
    g = 1.0 - 1.0 / np.sqrt(2.0)
    d = 1.0 - 1.0 / (2.0 * g)
    A_im = np.array([[0, 0, 0], [0, g, 0], [0, 1 - g, g]], float)
    A_ex = np.array([[0, 0, 0], [g, 0, 0], [d, 1 - d, 0]], float)
    return Tableau('ARS222', A_ex, A_ex[-1].copy(), A_im, A_im[-1].copy(),
                   np.array([0.0, g, 1.0]))


def ars343_gamma():
    """The root in (0, 1) of 6 g^3 - 18 g^2 + 9 g - 1 = 0 (the L-stable 3-stage SDIRK
    diagonal), g = 0.4358665215..."""
    r = np.roots([6.0, -18.0, 9.0, -1.0])
    r = np.real(r[(np.abs(np.imag(r)) < 1e-12) & (np.real(r) > 0.3) & (np.real(r) < 0.5)])
    g = float(r[0])
    for _ in range(3):                           # polish with Newton
        g -= (6 * g ** 3 - 18 * g ** 2 + 9 * g - 1) / (18 * g ** 2 - 36 * g + 9)
    return g


def ars343():
    g = ars343_gamma()
    b1 = -1.5 * g * g + 4.0 * g - 0.25
    b2 = 1.5 * g * g - 5.0 * g + 1.25
    A_im = np.array([[0, 0, 0, 0],
                     [0, g, 0, 0],
                     [0, (1 - g) / 2, g, 0],
                     [0, b1, b2, g]], float)
    # explicit coefficients as published (10 significant digits)
    A_ex = np.array([[0, 0, 0, 0],
                     [g, 0, 0, 0],
                     [0.3212788860, 0.3966543747, 0, 0],
                     [-0.105858296, 0.5529291479, 0.5529291479, 0]], float)
    b = np.array([0.0, b1, b2, g])
    return Tableau('ARS343', A_ex, b.copy(), A_im, b.copy(), np.array([0, g, (1 + g) / 2, 1.0]))


def imex_euler():
    """Tab. butcher_tableau_imex_euler."""
    return Tableau('IMEX_EULER', np.array([[0, 0], [1, 0]], float), np.array([1.0, 0.0]),
                   np.array([[0, 0], [0, 1]], float), np.array([0.0, 1.0]), np.array([0.0, 1.0]))


def ssp2_332():
    """Tab. butcher_tableau_ssp2_332. The printed c column (0, 1, 1/2) does not match the
    explicit row sums (1/2, 1); the row sums are taken: c = (0, 1/2, 1). Its implicit tableau
    has a non-zero first column, outside the form Alg. 1 assumes."""
    A_ex = np.array([[0, 0, 0], [0.5, 0, 0], [0.5, 0.5, 0]])
    A_im = np.array([[0.25, 0, 0], [0, 0.25, 0], [1 / 3, 1 / 3, 1 / 3]])
    b = np.array([1 / 3, 1 / 3, 1 / 3])
    return Tableau('SSP2_332', A_ex, b.copy(), A_im, b.copy(), np.array([0.0, 0.5, 1.0]))


def ssp3_433():
    """Tab. butcher_tableau_ssp3_433 (implicit first column non-zero, see ssp2_332)."""
    al, be, et = 0.24169426078821, 0.06042356519705, 0.12915286960590
    de = 0.5 - al - be - et
    A_ex = np.array([[0, 0, 0, 0], [0, 0, 0, 0], [0, 1, 0, 0], [0, 0.25, 0.25, 0]])
    A_im = np.array([[al, 0, 0, 0], [-al, al, 0, 0], [0, 1 - al, al, 0], [be, et, de, al]])
    b = np.array([0, 1 / 6, 1 / 6, 2 / 3])
    return Tableau('SSP3_433', A_ex, b.copy(), A_im, b.copy(), np.array([0, 0, 1, 0.5]))


TABLEAUS = {t().name: t for t in (ars222, ars343, imex_euler, ssp2_332, ssp3_433)}
