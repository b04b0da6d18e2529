"""The JSON-lines diagnostics log round-trips its records (no GPU needed)."""
import pytest

torch = pytest.importorskip("torch")
from paper_2602_13385_gb300 import diagnostics  # noqa: E402


def test_jsonl_round_trip(tmp_path):
    recs = [{"t": 0.5, "progenitor": 0, "E": -0.25, "lagrange_radii": {"0.5": 0.77}},
            {"t": 0.5, "progenitor": 1, "E": -0.2, "R": [1.0, 2.0, 3.0]}]
    path = str(tmp_path / "d.jsonl")
    with diagnostics.JsonlLog(path) as log:
        log.write(recs)
    with diagnostics.JsonlLog(path) as log:        # appends
        log.write(recs[:1])
    assert diagnostics.read_jsonl(path) == recs + recs[:1]
