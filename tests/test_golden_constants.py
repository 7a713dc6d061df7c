"""The oracle's constants against the values the paper prints."""
import json
import os

from oracle.constants import GAMMA


def test_gamma_matches_paper():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    assert GAMMA == gold["gamma_m_per_As"]["value"]
