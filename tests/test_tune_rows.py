"""Host logic of the selector driver: timed rows combined from several files with dtype
filters (the FP64 rows of one run with the split-precision rows of another)."""
import json

import pytest

from paper_1605_01078_gb300 import tune


def test_load_rows_combines_files_and_filters_dtypes(tmp_path):
    a = [{"m": 1, "n": 2, "k": 3, "dtype": 0, "times": [1.0]}, {"m": 4, "n": 5, "k": 6, "dtype": 2, "times": [2.0]}]
    b = [{"m": 7, "n": 8, "k": 9, "dtype": 2, "times": [3.0]}]
    pa, pb = tmp_path / "a.json", tmp_path / "b.jsonl"
    pa.write_text(json.dumps(a))
    pb.write_text("\n".join(json.dumps(r) for r in b) + "\n")
    assert tune.load_rows(str(pa)) == a
    assert tune.load_rows(f"{pa}:f64,{pb}") == [a[0]] + b
    assert tune.load_rows(f"{pa}:oz_bf16,{pb}:oz_bf16") == [a[1]] + b
    with pytest.raises(ValueError):
        tune.load_rows(f"{pa}:int8")
