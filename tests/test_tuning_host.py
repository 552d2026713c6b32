"""The autotuner's tables on the host (no GPU): the committed GB300 table
parses into a valid launch configuration, and a table written before a
setting existed falls back to the library default for it."""
import json
import os

import pytest

pytest.importorskip("torch")
import paper_1905_02082_gb300.refusion as R  # noqa: E402


def _load(monkeypatch, path):
    monkeypatch.setattr(R, "tuning_path", lambda device=None: path)
    monkeypatch.setattr(R, "_tuned", {})
    return R.tuned_launch_config()


def test_committed_gb300_table_is_valid(monkeypatch):
    path = os.path.join(R.TUNING_DIR, "NVIDIA_GB300_152sm.json")
    table = json.load(open(path))
    assert table["sm_count"] == 152 and set(table["launch"]) == {k for k, _ in R.rf_launch_config._fields_}
    cfg = _load(monkeypatch, path)
    assert all(getattr(cfg, k) == v for k, v in table["launch"].items())
    assert cfg.integrate_ctas_per_sm > 0 and cfg.cull_ctas_per_sm > 0 and cfg.fixup_ctas_per_sm > 0
    assert cfg.raycast_ctas_per_sm > 0 and cfg.batch_group >= 0


def test_missing_settings_take_the_defaults(monkeypatch, tmp_path):
    p = tmp_path / "old.json"
    p.write_text(json.dumps({"launch": {"integrate_ctas_per_sm": 12, "cull_ctas_per_sm": 4,
                                        "fixup_ctas_per_sm": 1}}))
    cfg = _load(monkeypatch, str(p))
    assert (cfg.integrate_ctas_per_sm, cfg.cull_ctas_per_sm, cfg.fixup_ctas_per_sm) == (12, 4, 1)
    assert (cfg.raycast_ctas_per_sm, cfg.batch_group) == (8, 16)
    assert _load(monkeypatch, str(tmp_path / "absent.json")) is None
