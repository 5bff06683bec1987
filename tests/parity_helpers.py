"""Helpers of the GPU parity tests: the moment error metric (the package's
metrics module, also used by the benchmark's FP32-vs-FP64 check) and the
oracle's moments of a state."""
from paper_1905_04597_gb300.metrics import rel_errors, term_scales  # noqa: F401


def oracle_moments(o, X):
    """(moments, streamed populations) of the oracle state X."""
    F = o.stream(X)
    return o.macro(F), F
