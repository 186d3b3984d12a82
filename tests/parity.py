"""Comparison used by every GPU parity assertion (imported by the test modules; not collected).

rel(a, b) is the larger of
  * the norm-wise relative difference ||a - b||_2 / ||b||_2, and
  * the element-wise one, max_i |a_i - b_i| / (ELEM_FACTOR * max_i |b_i|),
so that an assertion rel(a, b) <= tol also bounds every single element:
max_i |a_i - b_i| <= ELEM_FACTOR * tol * ||b||_inf.

Why both: at 4095^2 a norm-wise bound alone lets one wrong point carry sqrt(N) = 4095 times the
bound (one wrong row of a tile edge about 64 times). A rounding difference between two correct
computations is spread over the grid like the field itself: its max/RMS ratio is that of a smooth
field (2 to 4), while ||b||_inf >= RMS(b), so ELEM_FACTOR = 10 leaves such differences inside the
element-wise bound whenever they are inside the norm-wise one, and a localised error (a wrong
point, row, column or tile edge, whose max/RMS ratio grows with the grid) fails it.
"""
import numpy as np

ELEM_FACTOR = 10.0


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_elem(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if np.size(b) else 0.0


def rel(a, b):
    return max(rel_l2(a, b), rel_elem(a, b) / ELEM_FACTOR)
