"""The values the paper prints (tests/golden/paper_printed_values.txt, each with its table or
section) against what the oracle and the library take from them: the rotor model's bounds and
the paper cost form's safety distance (Table I), the temperature of the configured workload
inside the paper's range (Table I), and the gate frame's opening and outer widths (Sec. V),
checked through the oracle's exact frame SDF at points whose distance the printed widths fix.
Values the build deliberately takes from the workload instead (dt = 0.02 s, body rates within
8 rad/s, latents of 64 numbers, K x H of the benchmark) are listed but not asserted."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import gate_sdf as G

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_printed_values.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, value, _unit, source = (f.strip() for f in line.split("|"))
        assert source, name                    # every value cites where the paper prints it
        out[name] = float(value)
    return out


def test_every_value_has_a_citation_and_parses():
    g = _golden()
    assert len(g) >= 10 and g["rollouts_M"] == 8192 and g["horizon_K"] == 20


def test_rotor_model_bounds_are_the_printed_ones():
    g = _golden()
    p = W.rotor_params(64, 10)
    assert p["tdot_max"] == g["thrust_rate_max"] == -g["thrust_rate_min"]
    assert p["rotor_thrust_max"] == g["rotor_thrust_max"] and g["rotor_thrust_min"] == 0.0


def test_paper_cost_form_uses_the_printed_safety_distance_and_lambda_range():
    g = _golden()
    assert W.paper_params(64, 10)["d_safe"] == g["d_safe"]
    lam = W.params(64, 10)["lam"]
    assert g["lambda_min"] <= lam <= g["lambda_max"]


def test_library_defaults_match_the_printed_values():
    pytest.importorskip("ctypes")
    from paper_2603_07199_gb300 import binding as B
    try:
        cfg = B.mppi_config_default()
    except OSError:
        pytest.skip("library not built")
    g = _golden()
    assert cfg.tdot_max == pytest.approx(g["thrust_rate_max"])
    assert cfg.rotor_thrust_max == pytest.approx(g["rotor_thrust_max"])
    assert 2 * cfg.gate_inner_half == pytest.approx(g["gate_inner_width"])
    assert 2 * cfg.gate_outer_half == pytest.approx(g["gate_outer_width"])
    f32 = np.float32                           # the config holds float32 values
    assert f32(g["lambda_min"]) <= f32(cfg.lam) <= f32(g["lambda_max"])


def test_gate_frame_widths_through_the_oracle_sdf():
    """Opening width 1.0 m: the centre of the opening is 0.5 m from the frame and the SDF is
    zero at the opening's edge; outer width 1.5 m: the SDF is zero on the outer edge in the frame
    plane and grows with the distance beyond it."""
    g = _golden()
    a_in, a_out = g["gate_inner_width"] / 2, g["gate_outer_width"] / 2
    pts = np.array([[0.0, 0.0, 0.0],            # centre of the opening
                    [0.0, a_in, 0.0],           # edge of the opening
                    [0.0, a_out, 0.0],          # outer edge
                    [0.0, a_out + 0.25, 0.0],   # 0.25 m beyond the outer edge
                    [0.0, 0.0, -a_in + 0.1]])   # inside the opening, 0.1 m from its lower edge
    s = G.frame_sdf(pts)
    np.testing.assert_allclose(s, [a_in, 0.0, 0.0, 0.25, 0.1], atol=1e-12)
