"""Both instantiations of the binary forward kernel in one call (file named
to run after the other GPU files, so that under -x a failure here still
leaves their results)."""
import numpy as np
import pytest

from paper_2510_02639_gb300 import inputs as I
from tests.test_gpu_parity import G, assert_parity, assert_status, run_gpu  # noqa: F401 (G is a fixture)

pytestmark = pytest.mark.gpu


def test_mixed_laws_in_one_batch(G, oracle_mod):
    """One call over interleaved sets of different laws (linear; half-integer
    powers; a dark spot; quadratic; integer powers only; a bright spot): the
    binary forward call runs the linear and the generic instantiation of the
    kernel, each skipping the other's sets.  40 consecutive epochs per set
    (320 tiles, so blocks carry warm starts across several epochs and
    across set boundaries): every (set, epoch) against the oracle at 1e-5
    with the same status bits, and the pure-linear sets bitwise equal to the
    same batch with every set linear (the other sets' laws do not touch
    them)."""
    params, t = I.binary_batch()
    laws = [{}, dict(u1=0.2, a1=0.3, a3=-0.1), dict(spot_x=0.3, spot_y=-0.2, spot_r=0.4, spot_c=0.5),
            dict(u2=0.2), {}, dict(a2=0.3, a4=0.1), dict(spot_x=-0.2, spot_y=0.1, spot_r=0.3, spot_c=-0.5), {}]
    sets = [3, 11, 19, 27, 35, 43, 51, 59]
    mixed = [dict(params[s_], **law) for s_, law in zip(sets, laws)]
    plain = [params[s_] for s_ in sets]
    tt = np.stack([t[s_, 4980:5020] for s_ in sets])
    g = I.grid()
    A, st = run_gpu(G, mixed, tt, g)
    Ao, so = oracle_mod.magnification(mixed, tt, g)
    assert_parity(A, Ao, what="mixed laws")
    assert_status(st, so, what="mixed laws")
    Ap, sp = run_gpu(G, plain, tt, g)
    for k in (0, 4, 7):
        np.testing.assert_array_equal(A[k], Ap[k])
        np.testing.assert_array_equal(st[k], sp[k])
    assert not np.array_equal(A[2], Ap[2]) and not np.array_equal(A[1], Ap[1])
