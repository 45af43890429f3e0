"""The tools that choose the stored queries and write the stored oracle
counts (tests/golden/make_queries.py, make_expected.py): plan helpers, the
merge of partial selection files, and the consistency of the committed
query files with the rules they state.  CPU only; no oracle search runs."""
import json
import os
import sys

import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLD)
import make_queries as MQ  # noqa: E402


def test_interleave_alternates_then_appends_the_rest():
    assert MQ.interleave([1, 2, 3], ["a"]) == [1, "a", 2, 3]
    assert MQ.interleave([], ["a", "b"]) == ["a", "b"]
    assert MQ.interleave([1], [2]) == [1, 2]


def test_passed_over_cap_by_size():
    spec = {"max_passed": 8, "max_passed_by_size": {7: 24}}
    assert MQ.max_passed_for(spec, 6) == 8
    assert MQ.max_passed_for(spec, 7) == 24
    assert MQ.max_passed_for({}, 6) is None


def _query(q, att, kind):
    return {"labels": [att % 5] * q, "edges": [[i, i + 1] for i in range(q - 1)] + [[0, att + q]], "kind": kind,
            "attempt": att}


def _partial(path, kind, q, atts, log):
    d = {"workload": "mid", "graph_digest": "x", "selection_batch_updates": 10, "rule": "old text",
         "rejected": {"%s:%d" % (kind, q): {"stale": 99}},
         "chosen": {"%s:%d" % (kind, q): [_query(q, a, kind) for a in atts]},
         "rejections": {"%s:%d" % (kind, q): log}, "complete": False}
    with open(path, "w") as f:
        json.dump(d, f)


def test_merge_takes_the_plan_counts_and_recounts_rejections(tmp_path):
    spec = dict(MQ.SPECS["mid"])
    spec["plan"] = [("sparse", 5), ("dense", 6), ("sparse", 5)]
    _partial(tmp_path / "queries_t.sparse.q5.partial", "sparse", 5, [1, 4, 9],
             [[0, "r1"], [2, "r1"], [3, "r2"], [5, "r1"], [6, "r2"]])
    _partial(tmp_path / "queries_t.dense.q6.partial", "dense", 6, [2], [[0, "r2"], [1, "r2"]])
    out = MQ.merge("t", here=str(tmp_path), spec=spec)
    assert [(d["kind"], len(d["labels"]), d["attempt"]) for d in out["queries"]] == [
        ("sparse", 5, 1), ("dense", 6, 2), ("sparse", 5, 4)]
    # rejections before the last query used (attempt 4 for sparse:5, 2 for dense:6)
    assert out["rejected"]["sparse:5"] == {"r1": 2, "r2": 1, "attempts": 5}
    assert out["rejected"]["dense:6"] == {"r2": 2, "attempts": 3}
    assert out["rule"] == MQ.rule_text(spec)
    with open(tmp_path / "queries_t.json") as f:
        assert json.load(f)["queries"] == out["queries"]


def test_merge_refuses_too_few_and_duplicates(tmp_path):
    spec = dict(MQ.SPECS["mid"])
    spec["plan"] = [("sparse", 5)] * 4
    _partial(tmp_path / "queries_t.sparse.q5.partial", "sparse", 5, [1, 4, 9], [])
    with pytest.raises(SystemExit, match="the plan needs 4"):
        MQ.merge("t", here=str(tmp_path), spec=spec)
    spec["plan"] = [("sparse", 5), ("dense", 5)]
    _partial(tmp_path / "queries_t.dense.q5.partial", "dense", 5, [1], [])
    with open(tmp_path / "queries_t.dense.q5.partial") as f:
        d = json.load(f)
    d["chosen"]["dense:5"][0]["kind"] = "sparse"  # the same labels and edges as sparse attempt 1
    with open(tmp_path / "queries_t.dense.q5.partial", "w") as f:
        json.dump(d, f)
    with pytest.raises(SystemExit, match="same query twice"):
        MQ.merge("t", here=str(tmp_path), spec=spec)


@pytest.mark.parametrize("name", sorted(MQ.SPECS))
def test_stored_queries_follow_their_plan_and_rule(name):
    with open(os.path.join(GOLD, "queries_%s.json" % name)) as f:
        d = json.load(f)
    assert [(q["kind"], len(q["labels"])) for q in d["queries"]] == list(MQ.SPECS[name]["plan"])
    assert d["rule"] == MQ.rule_text(MQ.SPECS[name])
    keys = [json.dumps([q["labels"], q["edges"]]) for q in d["queries"]]
    assert len(set(keys)) == len(keys)


@pytest.mark.parametrize("name", ["large", "mid", "batched", "served"])
def test_stored_counts_belong_to_the_stored_queries(name):
    import make_expected as ME
    with open(os.path.join(GOLD, "expected_%s.json" % name)) as f:
        ex = json.load(f)
    assert ex["queries_digest"] == ME.file_digest(os.path.join(GOLD, "queries_%s.json" % name))
    nq = len(MQ.SPECS[name]["plan"])
    for b in ex["batches"]:
        n = len(b["count"])
        assert n == len(b["query"]) == len(b["update"]) == len(b["heavy"]) and n > 0
        assert all(0 <= j < nq for j in b["query"]) and all(0 <= u < b["updates"] for u in b["update"])
        pairs = list(zip(b["query"], b["update"]))
        assert len(set(pairs)) == len(pairs)
        assert not set(map(tuple, b["passed_over"])) & set(pairs)
