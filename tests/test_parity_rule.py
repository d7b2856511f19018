"""Why the GPU parity bar is calibrated instead of a flat 1e-10 on every
iterate (CPU, the oracle alone). On the 2,000 x 2,000 system the solve
takes 64 updates to 1e-10. Re-running the oracle on b (1 + 2^-50) and on
b (1 - 2^-50) moves b by a few units in its last place, a perturbation the
size of rounding (the scaled problems have exactly scaled solutions), yet,
like every Lanczos-type
recursion (Theorem 4.1's short recurrence relies on an orthogonality that
rounding erodes), its scalars leave 1e-10 of the unperturbed run after about
30 updates and end far apart, while x_64 still agrees to ~1e-8. No
implementation whose sums round differently from the oracle's can hold
every iterate to 1e-10, so the bar is 1e-10 while this spread allows it and
a fixed multiple of the spread afterwards."""
import numpy as np
import pytest

import oracle
from paper_2207_07615_gb300 import synth
from tests import _parity


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


@pytest.mark.parametrize("f", [1.0 + 2.0 ** -50, 1.0 - 2.0 ** -50])
def test_rounding_alone_moves_late_iterates_beyond_1e10(f):
    A, b, xs = synth.square_diag_dominant()
    K = 64
    r1 = oracle.residual(A, b, tol=0.0, maxit=K, hist=K)
    r2 = oracle.residual(A, b * f, tol=0.0, maxit=K, hist=K)
    h = r2["hist_s"].copy()
    h[:, [0, 1, 4]] /= f * f                     # rho, phi, theta scale with b^2; beta, gamma do not
    ds = _parity.rel_rows(h, r1["hist_s"])
    dx = _parity.rel_vec_rows(r2["hist_x"] / f, r1["hist_x"])
    # the leading updates agree to rounding level ...
    assert ds[:10].max() < 1e-12 and dx[:10].max() < 1e-12
    # ... later ones do not, in the scalars and in x_k
    first_s = int(np.argmax(ds > 1e-10)) + 1
    first_x = int(np.argmax(dx > 1e-10)) + 1
    assert ds.max() > 1e-3 and 20 <= first_s <= 45
    assert dx.max() > 1e-10 and 20 <= first_x <= 50
    # while the answer stays close to the unperturbed one and to x*
    assert dx[-1] < 1e-7
    assert np.linalg.norm(r2["x"] / f - xs) / np.linalg.norm(xs) < 1e-8
