"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This package only builds graphs (CSR arrays) and random label vectors from a
seed. It holds none of the method's arithmetic: no objectives, no operators,
no sorting and no random-number stream of the method. Both the CPU oracle
(``oracle/``) and the CUDA path (``paper_2506_01752_gb300``) consume what it
produces, and neither of them imports the other.

``synth.quality`` scores a detected partition against the planted ground
truth (NMI, AMI, pairwise F1); it is imported on its own and only by the tests
and the benchmark.
"""
from .graphs import (  # noqa: F401
    csr_from_edges,
    planted_partition,
    lfr_style,
    random_labels,
    batch_instances,
    serving_pool,
    workload,
    WORKLOADS,
)
