"""Measured errors of the CUDA path against the float64 oracle, kept as a record.

record(case, **errors) prints one line; when the environment variable
TM_ERROR_LOG names a file, it also appends the line there as JSON, so that a run
of the GPU tests leaves the table of measured errors per workload behind.
"""

import json
import os


def record(case, **errors):
    line = {"case": case, **{k: float(v) for k, v in errors.items()}}
    print("measured error:", json.dumps(line))
    path = os.environ.get("TM_ERROR_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")
