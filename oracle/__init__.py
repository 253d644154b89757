"""FP64 CPU oracle for the cue field and growth-cone step.

Test infrastructure only: the test suite, the smoke check and the CPU-baseline
leg of ``bench.py`` may import this package; the product library never does.
"""
from .oracle import (  # noqa: F401
    Grid,
    Cone,
    build,
    set_threads,
    philox4x32_10,
    noise,
    node_gradient,
    gradient_at,
    value_at,
    snr,
    field_step,
    field_window,
    cone_step,
    run,
    endpoint_loss,
    adjoint,
    adjoint_from_states,
    bin_points,
    connect,
    csr,
    bfs,
)
