"""Named configurations: every entry validates and its mesh builds (CPU)."""
import json

import numpy as np
import pytest

from paper_2509_01099_gb300 import configs as C


@pytest.mark.parametrize("name", list(C.CONFIGS))
def test_named_configs_validate_and_build_meshes(name):
    cfg = C.load_config(name)
    xi = C.mesh(cfg)
    assert xi.shape == (cfg["n"] + 2,) and np.all(np.diff(xi) > 0)


def test_json_round_trip_and_errors(tmp_path):
    p = tmp_path / "c.json"
    p.write_text(json.dumps({"dim": 2, "n": 32, "mesh": "erf", "Ra": 1e5}))
    cfg = C.load_config(str(p))
    assert cfg["Pr"] == 0.71 and cfg["precision"] == "fp32"
    for bad in ({"dim": 4, "n": 32, "mesh": "erf", "Ra": 1e5}, {"n": 32, "mesh": "erf", "Ra": 1e5},
                {"dim": 2, "n": 32, "mesh": "cosine", "Ra": 1e5},
                {"dim": 2, "n": 32, "mesh": "erf", "Ra": -1.0}):
        with pytest.raises(ValueError):
            C.validate(bad)
