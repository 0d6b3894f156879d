"""Host-side pieces of bench.py that need no GPU: the source laws that
--law applies and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_source_laws_are_valid_profiles():
    """Every law of inputs.SOURCE_LAWS, applied to every set of the headline
    batch, is a physical source: the brightness
    1 - u1 (1 - mu) - u2 (1 - mu)^2 - sum_k a_k (1 - mu^(k/2)) is
    non-negative on mu in [0, 1], its flux normalisation
    1 - u1/3 - u2/6 - sum_k a_k k/(k+4) is positive, and a spot lies inside
    the disk with contrast below 1 (else the magnification is NaN)."""
    from paper_2510_02639_gb300 import inputs as I
    params, _ = I.binary_batch()
    mu = np.linspace(0.0, 1.0, 2001)
    assert set(I.SOURCE_LAWS) == {"linear", "quadratic", "power4", "spot"}
    for name, law in I.SOURCE_LAWS.items():
        for p0 in params:
            p = dict(p0, **law)
            a = [p.get("a%d" % k, 0.0) for k in range(1, 5)]
            u1, u2 = p["u1"], p.get("u2", 0.0)
            I_mu = (1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2
                    - sum(a[k - 1] * (1.0 - mu ** (k / 2.0)) for k in range(1, 5)))
            assert I_mu.min() >= 0.0, (name, p0["u1"])
            assert 1.0 - u1 / 3.0 - u2 / 6.0 - sum(a[k - 1] * k / (k + 4.0) for k in range(1, 5)) > 0.0
            if p.get("spot_c", 0.0) != 0.0:
                assert np.hypot(p["spot_x"], p["spot_y"]) + p["spot_r"] <= 1.0 and p["spot_c"] < 1.0


def test_reference_arm_line_with_a_law():
    """bench.py --impl reference --law power4 runs the oracle on a tiny sample
    and prints one JSON line that names the law and carries the reference
    arm's keys."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--law", "power4",
                        "--steps", "1", "--warmup", "0", "--ref-sample", "2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "magnifications/s"
    assert d["config"]["law"] == "power4" and d["config"]["law_params"]["a1"] == 0.6
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
