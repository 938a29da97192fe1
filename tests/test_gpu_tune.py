"""The autotuner of the two-site split (mps_tune_two_site, MPS_FLAG_AUTOTUNE).

The tuner only chooses among configurations that are all correct, so parity is
checked against the oracle under every candidate (panel width x CTA count of the
pivoted panel kernel), and the tuner itself is checked for what it promises: a
candidate from the set, no slower than the defaults, a cache hit afterwards, a JSON
line in the file named by MPS_TUNE_CACHE, and handles that use the choice.
"""

import json

import numpy as np
import pytest

from oracle import mps as omps
from workloads import circuits, gates, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def gpu_mps(*a, **k):
    from paper_2505_06119_gb300 import MPS

    return MPS(*a, **k)


def sms():
    import torch

    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("nb", [8, 16, 32])
@pytest.mark.parametrize("frac", [1.0, 0.75, 0.5])
def test_every_candidate_matches_the_oracle(nb, frac):
    """A truncated 14-qubit brick-wall (FP64, canonical policy) with each tuner
    candidate forced through the configuration: the state equals the oracle's."""
    ctas = max(1, int(sms() * frac))
    ops = circuits.brickwall(14, 8, seed=19)
    ref = omps.OracleMPS(14, 16, "canon")
    ref.run(ops)
    with gpu_mps(14, 16, precision="fp64", panel_width=nb, debug_max_ctas=ctas) as m:
        m.run(ops)
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        rng = np.random.default_rng(nb)
        for _ in range(16):
            bits = rng.integers(0, 2, 14)
            assert abs(m.amplitude(bits) - ref.amplitude(bits)) < 1e-10


@pytest.mark.parametrize("nb", [8, 16])
def test_single_split_with_narrow_panels_matches_oracle(nb):
    """A single split on saturated sites (several panels of width nb) element by element."""
    from oracle import qr as oqr

    rng = np.random.default_rng(60 + nb)
    cl = cm = cr = chi = 96
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    with gpu_mps(18, 128, precision="fp64", policy="local", panel_width=nb) as m:
        m.set_site(8, a)
        m.set_site(9, b)
        m.apply_2q(8, g, chi)
        qa, rb = m.get_site(8), m.get_site(9)
    x = (a.reshape(2 * cl, cm) @ b.reshape(cm, 2 * cr)).reshape(cl, 2, 2, cr)
    theta = np.einsum("abcd,lcdr->labr", g.reshape(2, 2, 2, 2), x).reshape(2 * cl, 2 * cr)
    q, r, p, _ = oqr.cpqr(theta, kmax=chi)
    right = np.zeros((chi, 2 * cr), dtype=np.complex128)
    right[:, p] = r
    assert np.abs(qa.reshape(2 * cl, chi) - q).max() < 1e-10
    assert np.abs(rb.reshape(chi, -1) - right).max() < 1e-10 * np.abs(right).max()


def test_tuner_picks_a_candidate_and_caches_it(tmp_path, monkeypatch):
    from paper_2505_06119_gb300.mps import tune_two_site

    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("MPS_TUNE_CACHE", str(path))
    n_sm = sms()
    for prec in ("mixed", "fp64"):
        r = tune_two_site(prec, 200, 100, 160, 150, force=True)
        assert r["panel_width"] in (8, 16, 32)
        assert r["panel_ctas"] in (n_sm, max(1, n_sm * 3 // 4), max(1, n_sm // 2))
        assert r["candidates"] == 9
        assert 0 < r["ms"] <= 1.2 * r["default_ms"]
        again = tune_two_site(prec, 200, 100, 160, 150)
        assert again["candidates"] == 0
        assert (again["panel_width"], again["panel_ctas"]) == (r["panel_width"], r["panel_ctas"])
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 2
    assert {x["precision"] for x in lines} == {"c64", "c128"}
    assert all(x["m"] == 400 and x["n"] == 320 and x["k"] == 150 for x in lines)


def test_autotuned_handle_uses_the_choice_and_stays_correct():
    """A handle with MPS_FLAG_AUTOTUNE tunes each new split shape at its first split
    (outputs to scratch: the state is untouched), then splits with the choice: the
    panel launches of a split are ceil(k / chosen width), and the circuit still
    equals the oracle's."""
    from paper_2505_06119_gb300.mps import tune_two_site

    ops = circuits.brickwall(14, 8, seed=23)
    ref = omps.OracleMPS(14, 64, "local")
    ref.run(ops)
    with gpu_mps(14, 64, precision="fp64", policy="local", autotune=True) as m:
        m.run(ops)
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        rng = np.random.default_rng(2)
        for _ in range(16):
            bits = rng.integers(0, 2, 14)
            assert abs(m.amplitude(bits) - ref.amplitude(bits)) < 1e-10
    assert max(ref.bond_dims()) == 64  # splits above the one-CTA size were tuned
    # the choice for a 96 x 96 split with k = 48 is cached now; a profiled handle uses it
    choice = tune_two_site("fp64", 48, 48, 48, 48)
    with gpu_mps(14, 64, precision="fp64", policy="local", autotune=True, profile=True) as m:
        rng = np.random.default_rng(4)
        m.set_site(5, states.complex_gaussian(rng, (48, 2, 48)))
        m.set_site(6, states.complex_gaussian(rng, (48, 2, 48)))
        m.kernel_stats_reset()
        m.apply_2q(5, gates.haar_unitary(rng, 4), 48)
        st = m.kernel_stats()
    assert st["panel"]["launches"] == -(-48 // choice["panel_width"])
